"""GPU parity of the link Jacobians and the centre of mass (and its
Jacobian) against the oracle's dual-number differentiation of its own
forward kinematics, through the C ABI."""
import numpy as np
import pytest
import torch

from synthetic import inputs as I
from synthetic import robots as R
from tests import parity as PY

pytestmark = pytest.mark.gpu

ROBOTS = {"R7": R.r7, "R23": R.r23, "R48_payload": lambda: I.hand_payload(R.r48()),
          "mixed": R.mixed_joint_tree}


@pytest.fixture(scope="module")
def W():
    assert torch.cuda.is_available()
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe
    return wbe


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("rname", list(ROBOTS))
def test_jacobian_and_com_parity(W, O, rname):
    desc = ROBOTS[rname]()
    rob = W.Robot(desc, device=0)
    B = 45
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=PY.stable_seed(rname, 11))
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd))
    targets = sorted({0, desc.n // 2, desc.n - 1, 1 % desc.n})
    jac, com, jac_com = rob.kinematics(o["pose"], targets)
    torch.cuda.synchronize()
    rJ, rcom, rJc = O.kinematics(desc, q, targets)
    # velocities of points up to ~2 m from the joints: 1e-5 m per unit rate
    # times a few levels of rounding
    assert np.abs(jac.cpu().numpy() - rJ).max() <= 2e-5
    assert np.abs(com.cpu().numpy() - rcom).max() <= PY.POS_TOL
    assert np.abs(jac_com.cpu().numpy() - rJc).max() <= 2e-5
    # zero columns off the chain are exact zeros
    zero = rJ == 0.0
    assert (jac.cpu().numpy()[zero] == 0.0).all()


def test_outputs_each_alone_and_errors(W, O):
    desc = R.r23()
    rob = W.Robot(desc, device=0)
    q, qd, qdd = I.uniform_states(desc.dof, 33, seed=2)
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd))
    j1, c1, jc1 = rob.kinematics(o["pose"], [5, 9])
    j2, _, _ = rob.kinematics(o["pose"], [5, 9], com=False, jac_com=False)
    _, c3, _ = rob.kinematics(o["pose"], (), jac_com=False)
    _, _, jc4 = rob.kinematics(o["pose"], (), com=False)
    torch.cuda.synchronize()
    assert torch.equal(j1, j2) and torch.equal(c1, c3) and torch.equal(jc1, jc4)
    with pytest.raises(W.L.WbError) as ei:
        rob.kinematics(o["pose"], [desc.n])
    assert ei.value.code == W.L.WB_ERANGE
    with pytest.raises(W.L.WbError) as ei:
        rob.kinematics(o["pose"], list(range(65)) and [0] * 65)
    assert ei.value.code == W.L.WB_EINVAL


def test_full_size_humanoid_sampled(W, O):
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    B = 32768
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=1003)
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd))
    targets = [11, 27, 40, 48]
    jac, com, jac_com = rob.kinematics(o["pose"], targets)
    torch.cuda.synchronize()
    idx = np.array([0, 777, 20000, B - 1])
    rJ, rcom, rJc = O.kinematics(desc, q[:, idx], targets)
    assert np.abs(jac.cpu().numpy()[idx] - rJ).max() <= 2e-5
    assert np.abs(com.cpu().numpy()[idx] - rcom).max() <= PY.POS_TOL
    assert np.abs(jac_com.cpu().numpy()[idx] - rJc).max() <= 2e-5
