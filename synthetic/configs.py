"""The five benchmark workloads, by what they are and their sizes.

  small7    7-DoF chain, batch 64, forward (parity size)
  arm7      7-DoF chain, 4096 seeds x 32 timesteps, forward
  humanoid48  48-DoF tree, 1024 seeds x 32 timesteps, forward + backward
  uneven    256 x R7 + 256 x R23 + 256 x R48 problems, horizons U{16..64}
  trajopt48 48-DoF tree + 3 kg hand payloads, 512 seeds x 64 timesteps of
            B-spline states, cost gradient
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Workload:
    name: str
    robot: str
    batch: int
    seed: int
    backward: bool


SMALL7 = Workload("small7", "R7", 64, 1001, False)
ARM7 = Workload("arm7", "R7", 4096 * 32, 1002, False)
HUMANOID48 = Workload("humanoid48", "R48", 1024 * 32, 1003, True)
TRAJOPT48 = Workload("trajopt48", "R48", 512 * 64, 1005, True)

# trajopt48 B-spline shape
TRAJOPT_SEEDS = 512
TRAJOPT_STEPS = 64
TRAJOPT_KNOTS = 16
TRAJOPT_DT = 0.25
TORQUE_LIMIT = 30.0
COLLISION_WEIGHT = 1.0
ACTIVATION_DISTANCE = 0.02  # m, summed collision hinge of the trajopt48 variant
# motion terms of the trajopt48 loss (smooth |qdd|^2, length |qd|^2, energy
# sum (qd tau dt)^2), weighted so that each is of the order of a few hundred
# on the workload's states, like the torque hinges
SMOOTH_WEIGHT = 0.01
LENGTH_WEIGHT = 1.0
ENERGY_WEIGHT = 0.01
