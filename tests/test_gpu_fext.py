"""GPU parity with external link wrenches (f_ext): torques, the joint
gradients with f_ext present, and dL/df_ext = -fbar against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from synthetic import inputs as I
from synthetic import robots as R
from tests import parity as PY

pytestmark = pytest.mark.gpu

ROBOTS = {"R7": R.r7, "R23": R.r23, "R48": R.r48, "mixed": R.mixed_joint_tree}


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


def tunes(W):
    return {"tree1": W.Tune(kernel=3, lanes_per_config=1), "tree_auto": W.Tune(kernel=3),
            "plain": W.PLAIN}


@pytest.mark.parametrize("rname", list(ROBOTS))
@pytest.mark.parametrize("kname", ["tree1", "tree_auto", "plain"])
def test_fext_parity(W, O, rname, kname):
    desc = ROBOTS[rname]()
    rob = W.Robot(desc, device=0)
    B = 19 if rname == "R48" else 41
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=PY.stable_seed(rname, 13))
    rng = np.random.default_rng(PY.stable_seed(rname, 14))
    fext = rng.normal(scale=5.0, size=(B, desc.n, 6)).astype(np.float32)
    tune = tunes(W)[kname]
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=tune, f_ext=cuda(fext), dmin=False,
                 sphere=False)
    torch.cuda.synchronize()
    ref = O.evaluate(desc, q, qd, qdd, fext=fext.astype(np.float64), want=("tau",))
    tau, rtau = o["tau"].cpu().numpy(), ref["tau"]
    scale = np.maximum(np.abs(rtau).max(axis=0), 1.0)
    assert (np.abs(tau - rtau).max(axis=0) <= PY.TAU_REL * scale).all()
    gt = rng.normal(size=(desc.dof, B)).astype(np.float32)
    g_fext = torch.empty((B, desc.n, 6), device="cuda")
    g = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), None, None, None, None, cuda(gt),
                          tune=tune, f_ext=cuda(fext), g_fext=g_fext)
    torch.cuda.synchronize()
    rg = O.gradient(desc, q, qd, qdd, g_tau=gt, fext=fext.astype(np.float64))
    PY.check_gradient([x.cpu().numpy() for x in g], rg)
    rf = O.fext_gradient(desc, q, qd, qdd, fext.astype(np.float64), gt.astype(np.float64))
    gf = g_fext.cpu().numpy()
    for b in range(B):
        assert np.linalg.norm(gf[b] - rf[b]) <= PY.GRAD_REL * max(np.linalg.norm(rf[b]), 1e-6)


def test_support_forces_cancel_gravity_on_gpu(W, O):
    """Forces that hold every link up (computed from the GPU's own poses)
    leave ~zero torque at rest on the humanoid with payloads."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    B = 64
    q, _, _ = I.uniform_states(desc.dof, B, seed=5)
    z = np.zeros_like(q)
    o = rob.eval(cuda(q), cuda(z), cuda(z), dmin=False, sphere=False)
    P = o["pose"].cpu().numpy().astype(np.float64)
    f = np.zeros((B, desc.n, 6))
    pts = [(k, desc.mass[k], desc.com[k]) for k in range(desc.n)]
    pts += [(int(l), m, x) for l, m, x in zip(desc.pm_link, desc.pm_mass, desc.pm_pos)]
    g = np.asarray(desc.gravity, float)
    for k, m, x in pts:
        F = m * np.einsum("bji,j->bi", P[:, k, :9].reshape(B, 3, 3), -g)
        f[:, k, 3:] += F
        f[:, k, :3] += np.cross(np.broadcast_to(x, F.shape), F)
    o2 = rob.eval(cuda(q), cuda(z), cuda(z), f_ext=cuda(f), dmin=False, sphere=False)
    torch.cuda.synchronize()
    t0 = np.abs(o["tau"].cpu().numpy()).max()
    assert t0 > 10.0 and np.abs(o2["tau"].cpu().numpy()).max() < 1e-4 * t0


def test_fused_rejects_external_forces(W):
    desc = R.r7()
    rob = W.Robot(desc, device=0)
    q, qd, qdd = I.uniform_states(desc.dof, 8, seed=1)
    with pytest.raises(W.L.WbError) as ei:
        rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=W.FUSED,
                 f_ext=torch.zeros((8, desc.n, 6), device="cuda"))
    assert ei.value.code == W.L.WB_EINVAL
