"""GPU parity of the all-pairs summed self-collision hinge (cost and its
sphere-centre gradient, then dcost/dq through the backward sweep) against
the FP64 oracle, through the C ABI."""
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


_robots = {}


def robot(W, name):
    if name not in _robots:
        _robots[name] = (ROBOTS[name](), W.Robot(ROBOTS[name](), device=0))
    return _robots[name]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def pair_distances(O, desc, q):
    """Oracle sphere centres -> d_p [B][P] and active partners per sphere."""
    c = O.evaluate(desc, q, want=("sph",))["sph"]
    P = np.asarray(desc.pairs).reshape(-1, 2)
    rad = np.asarray(desc.sph_r, np.float64)
    nrm = np.linalg.norm(c[:, P[:, 0]] - c[:, P[:, 1]], axis=2)
    return nrm - rad[P[:, 0]] - rad[P[:, 1]], P


def check(desc, got_cost, got_g, ref_cost, ref_g, d, P, eta, w):
    """Per configuration, away from the kink: cost within the distance
    tolerance times the active pairs; each sphere's gradient within 1e-4 of
    w times its active partners (a unit vector per active pair)."""
    keep = ~(np.abs(d - eta) < 1e-5).any(axis=1)
    act = d < eta
    n_act = act.sum(axis=1)
    per_sphere = np.zeros((d.shape[0], desc.S))
    for k in range(P.shape[0]):
        per_sphere[:, P[k, 0]] += act[:, k]
        per_sphere[:, P[k, 1]] += act[:, k]
    tol_c = w * (PY.POS_TOL * n_act + 1e-6 * np.abs(ref_cost) + 1e-6)
    assert (np.abs(got_cost - ref_cost)[keep] <= tol_c[keep]).all()
    if got_g is not None:
        tol_g = 1e-4 * w * (per_sphere + 1.0)
        err = np.abs(got_g - ref_g).max(axis=2)
        assert (err[keep] <= tol_g[keep]).all()
    return keep.mean()


@pytest.mark.parametrize("rname", list(ROBOTS))
@pytest.mark.parametrize("eta", [0.0, 0.02, 0.1])
def test_hinge_parity(W, O, rname, eta):
    desc, rob = robot(W, rname)
    B = 61 if rname == "R48" else 203
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=PY.stable_seed(rname, 7))
    w = 1.3
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd))
    cost, g = rob.self_collision_hinge(o["pose"], eta, w)
    torch.cuda.synchronize()
    ref_cost, ref_g = O.pair_hinge(desc, q, eta, w)
    d, P = pair_distances(O, desc, q)
    kept = check(desc, cost.cpu().numpy(), g.cpu().numpy(), ref_cost, ref_g, d, P, eta, w)
    # a configuration is set aside when any of its pairs lies within 1e-5 m
    # of eta (there a float decides activity); with hundreds of pairs near
    # eta that is up to ~15 % of random configurations
    assert kept > 0.75
    # cost alone, no gradient buffer
    c2, g2 = rob.self_collision_hinge(o["pose"], eta, w, want_grad=False)
    torch.cuda.synchronize()
    assert g2 is None and torch.equal(c2, cost)


def test_hinge_hand_built_sliders(W):
    """Slider spheres at exact binary positions: the float kernel reproduces
    the hand values (see the oracle pin of the same case)."""
    radii = [0.25, 0.125, 0.5]
    n = 3
    desc = R._plain("sliders", [-1] * n, [R.PRISMATIC] * n, [[1, 0, 0]] * n,
                    [R._Tp(0, 0, 0)] * n, mass=[1.0] * n, com=np.zeros((n, 3)),
                    Icom=[[0.1, 0.1, 0.1, 0, 0, 0]] * n, sph_link=list(range(n)),
                    sph_c=np.zeros((n, 3)), sph_r=radii,
                    pairs=[[i, j] for i in range(n) for j in range(i + 1, n)])
    rob = W.Robot(desc, device=0)
    q = np.array([[0.0, 0.0], [0.375, 0.5], [0.5, 5.0]])  # two configurations
    o = rob.eval(cuda(q), cuda(np.zeros_like(q)), cuda(np.zeros_like(q)))
    cost, g = rob.self_collision_hinge(o["pose"], 0.125, 2.0)
    torch.cuda.synchronize()
    c, gg = cost.cpu().numpy(), g.cpu().numpy()
    # config 0: d = (0, -0.25, -0.5) -> 2 (0.125 + 0.375 + 0.625); config 1: d01 = 0.125 = eta
    assert c[0] == pytest.approx(2.0 * 1.125, abs=1e-6) and c[1] == 0.0
    assert np.allclose(gg[0, :, 0], [4.0, 0.0, -4.0], atol=1e-6)
    assert np.allclose(gg[1], 0.0) and np.allclose(gg[0, :, 1:], 0.0)


@pytest.mark.parametrize("rname", ["R7", "R48"])
def test_hinge_gradient_through_backward(W, O, rname):
    """dcost/dq: the sphere gradient fed to the backward sweep against the
    oracle's dual-number VJP of its own sphere gradient."""
    desc, rob = robot(W, rname)
    B = 37
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=99)
    eta, w = 0.03, 0.8
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd))
    _, g = rob.self_collision_hinge(o["pose"], eta, w)
    gq, gqd, gqdd = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), None, None, g, None, None)
    torch.cuda.synchronize()
    _, ref_g = O.pair_hinge(desc, q, eta, w)
    rq, rqd, rqdd = O.gradient(desc, q, qd, qdd, g_sph=ref_g)
    d, _ = pair_distances(O, desc, q)
    keep = ~(np.abs(d - eta) < 1e-5).any(axis=1)
    PY.check_gradient([gq.cpu().numpy(), gqd.cpu().numpy(), gqdd.cpu().numpy()],
                      (rq, rqd, rqdd), mask=keep)
    assert keep.mean() > 0.9


def test_hinge_full_size_humanoid_sampled_and_deterministic(W, O):
    desc, rob = robot(W, "R48")
    B = 32768
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=1003)
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd))
    eta, w = 0.02, 1.0
    cost, g = rob.self_collision_hinge(o["pose"], eta, w)
    cost2, g2 = rob.self_collision_hinge(o["pose"], eta, w)
    torch.cuda.synchronize()
    assert torch.equal(cost, cost2) and torch.equal(g, g2)
    idx = np.array([0, 1, 4095, 16384, B - 1])
    ref_cost, ref_g = O.pair_hinge(desc, q[:, idx], eta, w)
    d, P = pair_distances(O, desc, q[:, idx])
    check(desc, cost.cpu().numpy()[idx], g.cpu().numpy()[idx], ref_cost, ref_g, d, P, eta, w)


def test_hinge_without_pairs_and_over_two_chunks(W, O):
    """No masked pairs: zero cost and gradient.  The humanoid with every pair
    of links a joint apart masked in (39 rounds of 32 pair blocks, two
    chunks of the block walk) against the oracle."""
    desc = R.r7().with_pairs(np.zeros((0, 2), np.int32))
    rob = W.Robot(desc, device=0)
    q, qd, qdd = I.uniform_states(desc.dof, 45, seed=12)
    o = rob.eval(cuda(q), tau=False)
    cost, g = rob.self_collision_hinge(o["pose"], 0.05, 1.0)
    torch.cuda.synchronize()
    assert (cost.cpu().numpy() == 0.0).all() and (g.cpu().numpy() == 0.0).all()
    desc = R.r48(min_tree_dist=1)
    rob = W.Robot(desc, device=0)
    assert W.plan_info(desc)[1][3] == 39
    q, qd, qdd = I.uniform_states(desc.dof, 53, seed=13)
    o = rob.eval(cuda(q), tau=False)
    eta, w = 0.02, 0.7
    cost, g = rob.self_collision_hinge(o["pose"], eta, w)
    torch.cuda.synchronize()
    ref_cost, ref_g = O.pair_hinge(desc, q, eta, w)
    d, P = pair_distances(O, desc, q)
    kept = check(desc, cost.cpu().numpy(), g.cpu().numpy(), ref_cost, ref_g, d, P, eta, w)
    assert kept > 0.75
