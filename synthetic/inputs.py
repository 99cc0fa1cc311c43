"""Seeded synthetic inputs for the five benchmark workloads.

Input creation only: uniform joint states, random upstream gradients, random
B-spline control points, payload descriptions and the uneven-batch work mix.
No evaluation arithmetic lives here (the B-spline is evaluated by each side
from the control points this module draws).

All arrays are float32 (or int32) and use the library's layouts:
  q, qd, qdd, g_tau      [d][B]   joint-major, batch contiguous
  g_pose                 [B][n][12]
  g_sph                  [B][S][3]
  g_dmin                 [B]
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import robots as R


def uniform_states(dof: int, B: int, seed: int, q_range=np.pi, qd_range=2.0,
                   qdd_range=5.0):
    """q ~ U(-pi, pi), qd ~ U(-2, 2) rad/s, qdd ~ U(-5, 5) rad/s^2, i.i.d."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(-q_range, q_range, size=(dof, B)).astype(np.float32)
    qd = rng.uniform(-qd_range, qd_range, size=(dof, B)).astype(np.float32)
    qdd = rng.uniform(-qdd_range, qdd_range, size=(dof, B)).astype(np.float32)
    return q, qd, qdd


def upstream_grads(robot: R.Robot, B: int, seed: int, pose=True, sph=True, dmin=True,
                   tau=True):
    """Standard-normal upstream gradients for each output (None when off)."""
    rng = np.random.default_rng(seed)
    g_pose = rng.standard_normal((B, robot.n, 12)).astype(np.float32) if pose else None
    g_sph = rng.standard_normal((B, robot.S, 3)).astype(np.float32) if sph else None
    g_dmin = rng.standard_normal(B).astype(np.float32) if dmin else None
    g_tau = rng.standard_normal((robot.dof, B)).astype(np.float32) if tau else None
    return g_pose, g_sph, g_dmin, g_tau


def batch_columns(robot: R.Robot, lo: int, hi: int, seed: int, block: int = 32):
    """Columns [lo, hi) of one seeded batch of configurations: the states of
    uniform_states (same ranges) and the standard-normal upstream gradients of
    upstream_grads, drawn in blocks of `block` consecutive columns (one seed's
    timesteps), block k from the generator seeded with (seed, k).  Any
    contiguous slice is therefore the same whoever draws it: ranks that split
    one batch draw only their own columns.  Returns (q, qd, qdd, g_pose,
    g_sph, g_dmin, g_tau) in the library's layouts."""
    if not 0 <= lo <= hi:
        raise ValueError("bad column range [%d, %d)" % (lo, hi))
    k0, k1 = lo // block, (hi + block - 1) // block
    parts = [[] for _ in range(7)]
    for k in range(k0, k1):
        rng = np.random.default_rng([seed, k])
        d = robot.dof
        draws = (rng.uniform(-np.pi, np.pi, size=(d, block)),
                 rng.uniform(-2.0, 2.0, size=(d, block)),
                 rng.uniform(-5.0, 5.0, size=(d, block)),
                 rng.standard_normal((block, robot.n, 12)),
                 rng.standard_normal((block, robot.S, 3)),
                 rng.standard_normal(block),
                 rng.standard_normal((d, block)))
        for lst, x in zip(parts, draws):
            lst.append(x.astype(np.float32))
    a, b = lo - k0 * block, hi - k0 * block
    out = []
    for i, lst in enumerate(parts):
        if not lst:
            shape = {0: (robot.dof, 0), 1: (robot.dof, 0), 2: (robot.dof, 0),
                     3: (0, robot.n, 12), 4: (0, robot.S, 3), 5: (0,), 6: (robot.dof, 0)}[i]
            out.append(np.zeros(shape, np.float32))
            continue
        joint = i in (0, 1, 2, 6)
        x = np.concatenate(lst, axis=1 if joint else 0)
        out.append(np.ascontiguousarray(x[:, a:b] if joint else x[a:b]))
    return tuple(out)


def bspline_controls(dof: int, n_traj: int, K: int, seed: int, lim=np.pi / 2):
    """Control points U ~ U(-pi/2, pi/2), layout [n_traj][d][K]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-lim, lim, size=(n_traj, dof, K)).astype(np.float32)


def hand_payload(robot: R.Robot, mass: float = 3.0, pos=(0.0, 0.0, 0.05)) -> R.Robot:
    """The robot with a point payload of `mass` kg at `pos` (link frame) on each
    hand link."""
    hands = R.hand_links(robot)
    return robot.with_point_masses(hands, [mass] * len(hands), [pos] * len(hands))


@dataclass
class UnevenBatch:
    robots: list          # distinct robot models
    robot_of: np.ndarray  # [n_problems] index into robots
    horizon: np.ndarray   # [n_problems] configurations per problem


def uneven_mix(per_type: int = 256, seed: int = 4, h_lo: int = 16, h_hi: int = 64):
    """256 x R7 chains, 256 x R23 trees, 256 x R48 trees, horizons U{16..64},
    problems interleaved in a seeded random order."""
    rng = np.random.default_rng(seed)
    robots = [R.r7(), R.r23(), R.r48()]
    robot_of = np.repeat(np.arange(3, dtype=np.int32), per_type)
    rng.shuffle(robot_of)
    horizon = rng.integers(h_lo, h_hi + 1, size=robot_of.shape[0]).astype(np.int32)
    return UnevenBatch(robots, robot_of, horizon)
