"""GPU parity of the trajectory-optimisation ends: B-spline states and their
control-point gradient, the per-configuration cost, and the whole chain
U -> states -> whole-body evaluation -> cost -> dL/dU on the 48-DoF humanoid
with 3 kg hand payloads, against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from synthetic import configs as CF
from synthetic import inputs as I
from synthetic import robots as R
from tests import parity as PY

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("n_traj,d,K,T,dt", [(5, 7, 16, 64, 0.25), (3, 5, 6, 9, 0.3),
                                             (2, 3, 4, 2, 0.1), (1, 48, 40, 301, 0.05),
                                             (0, 4, 8, 16, 0.25)])
def test_bspline_forward_and_vjp(W, O, n_traj, d, K, T, dt):
    rng = np.random.default_rng(K * 100 + T)
    U = rng.uniform(-np.pi / 2, np.pi / 2, size=(n_traj, d, K)).astype(np.float32)
    q, qd, qdd = W.bspline_eval(cuda(U), T, dt)
    torch.cuda.synchronize()
    if n_traj == 0:
        return
    ref = O.bspline(U.astype(np.float64), T, dt)
    for got, r, order in zip((q, qd, qdd), ref, range(3)):
        scale = np.pi / dt ** order
        assert np.abs(got.cpu().numpy() - r).max() <= 2e-6 * scale
    g = [rng.normal(size=(d, n_traj * T)).astype(np.float32) for _ in range(3)]
    gU = W.bspline_backward(*[cuda(x) for x in g], n_traj, K, T, dt)
    torch.cuda.synchronize()
    Uref = O.bspline_vjp(*[x.astype(np.float64) for x in g], n_traj, K, T, dt)
    got = gU.cpu().numpy()
    for tr in range(n_traj):
        for j in range(d):
            e = np.abs(got[tr, j] - Uref[tr, j]).max()
            assert e <= 1e-5 * max(1.0, np.abs(Uref[tr, j]).max()) * (1 + T / K), (tr, j, e)
    # adjoint identity on the GPU's own results
    lhs = sum(float((a.double() * cuda(b).double()).sum()) for a, b in zip((q, qd, qdd), g))
    rhs = float((cuda(U).double() * gU.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + np.abs(got).sum())
    # one upstream gradient alone
    gq_only = W.bspline_backward(cuda(g[0]), None, None, n_traj, K, T, dt)
    ref_q = O.bspline_vjp(g[0].astype(np.float64), None, None, n_traj, K, T, dt)
    assert np.abs(gq_only.cpu().numpy() - ref_q).max() <= 1e-5 * max(1.0, np.abs(ref_q).max()) * T


@pytest.mark.parametrize("n_traj,d,K,T,dt", [(4, 7, 16, 64, 0.25), (3, 5, 1, 9, 0.3),
                                             (2, 3, 5, 40, 0.1), (1, 48, 13, 301, 0.05)])
@pytest.mark.parametrize("has_start,end_static", [(True, False), (False, True), (True, True)])
def test_bspline_boundary_conditions_match_oracle(W, O, n_traj, d, K, T, dt, has_start,
                                                  end_static):
    """Ghost knots from a start state and the static goal (Sec. 4.2): states,
    control-point gradient and start-state gradient against the oracle."""
    if K + 3 * has_start + 3 * end_static < 4:
        pytest.skip("fewer than 4 knots")
    rng = np.random.default_rng(K * 1000 + T + 7 * has_start + 3 * end_static)
    U = rng.uniform(-np.pi / 2, np.pi / 2, size=(n_traj, d, K)).astype(np.float32)
    start = rng.uniform(-1.0, 1.0, size=(n_traj, d, 3)).astype(np.float32) if has_start else None
    q, qd, qdd = W.bspline_eval(cuda(U), T, dt, start=None if start is None else cuda(start),
                                end_static=end_static)
    torch.cuda.synchronize()
    ref = O.bspline_bc(U.astype(np.float64), T, dt,
                       start=None if start is None else start.astype(np.float64),
                       end_static=end_static)
    for got, r, order in zip((q, qd, qdd), ref, range(3)):
        scale = np.pi / dt ** order
        assert np.abs(got.cpu().numpy() - r).max() <= 2e-6 * scale
    g = [rng.normal(size=(d, n_traj * T)).astype(np.float32) for _ in range(3)]
    gU, gs = W.bspline_backward_bc(*[cuda(x) for x in g], n_traj, K, T, dt, has_start=has_start,
                                   end_static=end_static)
    torch.cuda.synchronize()
    rU, rs = O.bspline_bc_vjp(*[x.astype(np.float64) for x in g], n_traj, K, T, dt,
                              has_start=has_start, end_static=end_static)
    Kx = K + 3 * has_start + 3 * end_static
    tol = 1e-5 * (1 + T / Kx) * max(1.0, np.abs(rU).max())
    assert np.abs(gU.cpu().numpy() - rU).max() <= tol * (4 if end_static else 1)
    if has_start:
        assert np.abs(gs.cpu().numpy() - rs).max() <= 1e-5 * (1 + T / Kx) * max(1.0, np.abs(rs).max())
    else:
        assert gs is None
    # the additive q-dot / q-ddot gradients join before the transpose
    gU2, _ = W.bspline_backward_bc(cuda(g[0]), None, None, n_traj, K, T, dt,
                                   has_start=has_start, end_static=end_static,
                                   gqd_add=cuda(g[1]), gqdd_add=cuda(g[2]), want_start=False)
    torch.cuda.synchronize()
    assert torch.equal(gU2, gU)


def test_bspline_boundary_first_sample_and_static_end(W):
    """Closed forms on the GPU: the first sample carries the start state one
    interval forward with zero jerk; with a static goal the final sample is
    the last control point at rest."""
    rng = np.random.default_rng(77)
    n_traj, d, K, T, dt = 8, 6, 10, 33, 0.25
    U = rng.uniform(-1.0, 1.0, size=(n_traj, d, K)).astype(np.float32)
    start = rng.uniform(-1.0, 1.0, size=(n_traj, d, 3)).astype(np.float32)
    q, qd, qdd = W.bspline_eval(cuda(U), T, dt, start=cuda(start), end_static=True)
    torch.cuda.synchronize()
    q, qd, qdd = (x.cpu().numpy().astype(np.float64) for x in (q, qd, qdd))
    th, v, a = (start[..., i].astype(np.float64) for i in range(3))
    first, last = np.arange(n_traj) * T, np.arange(n_traj) * T + T - 1
    assert np.allclose(q[:, first].T, th + v * dt + a * dt * dt / 2, atol=2e-6)
    assert np.allclose(qd[:, first].T, v + a * dt, atol=2e-5)
    assert np.allclose(qdd[:, first].T, a, atol=2e-4)
    assert np.allclose(q[:, last].T, U[..., -1], atol=2e-6)
    assert np.allclose(qd[:, last], 0.0, atol=2e-5) and np.allclose(qdd[:, last], 0.0, atol=2e-4)


def test_bspline_boundary_errors_and_determinism(W):
    rng = np.random.default_rng(5)
    x = cuda(rng.normal(size=(2, 3, 3)))
    with pytest.raises(W.L.WbError):  # 3 control points, no boundary knots
        W.bspline_eval(x, 8, 0.1)
    q, _, _ = W.bspline_eval(x, 8, 0.1, end_static=True)  # 6 knots: fine
    assert torch.isfinite(q).all()
    g = cuda(rng.normal(size=(3, 16)))
    with pytest.raises(W.L.WbError):  # a start-state gradient without a start state
        W.bspline_backward_bc(g, None, None, 2, 3, 8, 0.1, has_start=False, end_static=True,
                              g_start=torch.empty((2, 3, 3), device="cuda"))
    a = W.bspline_backward_bc(g, g, g, 2, 3, 8, 0.1, has_start=True, end_static=True)
    b = W.bspline_backward_bc(g, g, g, 2, 3, 8, 0.1, has_start=True, end_static=True)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_bspline_backward_is_deterministic(W):
    rng = np.random.default_rng(3)
    n_traj, d, K, T = 64, 48, 16, 64
    g = [cuda(rng.normal(size=(d, n_traj * T))) for _ in range(3)]
    a = W.bspline_backward(*g, n_traj, K, T, 0.25)
    b = W.bspline_backward(*g, n_traj, K, T, 0.25)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_trajopt_cost_matches_oracle_on_the_same_inputs(W, O):
    """Same float32 torques and distances on both sides: the hinge decisions
    and gradients are identical, the cost agrees to float rounding."""
    rng = np.random.default_rng(8)
    d, B = 48, 1000
    tau = rng.normal(scale=30.0, size=(d, B)).astype(np.float32)
    tau[0, :5] = [30.0, -30.0, 30.000002, -30.000002, 0.0]  # on and just past the limits
    dmin = rng.normal(scale=0.05, size=B).astype(np.float32)
    dmin[:3] = [0.0, -0.0, 1e-9]
    lo = np.full(d, -30.0, np.float32)
    hi = np.full(d, 30.0, np.float32)
    hi[3] = 25.0
    cost, g_tau, g_dmin = W.trajopt_cost(cuda(tau), cuda(dmin), cuda(lo), cuda(hi), 2.5)
    torch.cuda.synchronize()
    rc, rg, rm = O.trajopt_cost(tau, dmin, lo, hi, 2.5)
    assert np.array_equal(g_tau.cpu().numpy(), rg)
    assert np.array_equal(g_dmin.cpu().numpy(), rm)
    assert np.allclose(cost.cpu().numpy(), rc, rtol=2e-6, atol=1e-4)
    # distances only / torques only
    c2, _, gm2 = W.trajopt_cost(cuda(tau), None, cuda(lo), cuda(hi), 2.5)
    c3, _, _ = W.trajopt_cost(cuda(tau[:, :0]), None, cuda(lo), cuda(hi), 2.5)
    torch.cuda.synchronize()
    assert np.allclose(c2.cpu().numpy(), O.trajopt_cost(tau, np.ones(B), lo, hi, 0.0)[0],
                       rtol=2e-6, atol=1e-4)


def test_trajopt_cost_motion_terms_match_oracle(W, O):
    """wb_trajopt_cost_ext on the same float32 states and torques as the
    oracle: the smooth, length and energy terms and their direct gradients
    agree to float rounding, the hinge decisions are unchanged."""
    rng = np.random.default_rng(21)
    d, B = 48, 777
    tau = rng.normal(scale=30.0, size=(d, B)).astype(np.float32)
    qd = rng.normal(scale=3.0, size=(d, B)).astype(np.float32)
    qdd = rng.normal(scale=20.0, size=(d, B)).astype(np.float32)
    dmin = rng.normal(scale=0.05, size=B).astype(np.float32)
    lo, hi = np.full(d, -30.0, np.float32), np.full(d, 30.0, np.float32)
    kw = dict(smooth=0.01, length=1.0, energy=0.01, dt=0.05)
    got = W.trajopt_cost_ext(cuda(tau), cuda(dmin), cuda(qd), cuda(qdd), cuda(lo), cuda(hi), 2.5,
                             **kw)
    torch.cuda.synchronize()
    ref = O.trajopt_cost(tau, dmin, lo, hi, 2.5, qd, qdd, **kw)
    got = [g.cpu().numpy().astype(np.float64) for g in got]
    # each term is a sum of d float products: relative 1e-5 of its size
    mag = (kw["smooth"] * qdd.astype(np.float64) ** 2 + kw["length"] * qd.astype(np.float64) ** 2
           + kw["energy"] * kw["dt"] ** 2 * (qd.astype(np.float64) * tau) ** 2
           + np.abs(tau)).sum(axis=0) + 2.5 * np.abs(dmin)
    assert (np.abs(got[0] - ref[0]) <= 1e-5 * mag + 1e-5).all()
    for g, r in zip(got[1:], ref[1:]):
        assert np.allclose(g, r, rtol=1e-5, atol=1e-5 * np.abs(r).max())
    assert np.array_equal(got[2], ref[2])  # the collision hinge is untouched
    # zero motion weights: the plain cost, bit for bit
    c0 = W.trajopt_cost_ext(cuda(tau), cuda(dmin), cuda(qd), cuda(qdd), cuda(lo), cuda(hi), 2.5)
    c1 = W.trajopt_cost(cuda(tau), cuda(dmin), cuda(lo), cuda(hi), 2.5)
    torch.cuda.synchronize()
    for a, b in zip(c0[:3], c1):
        assert torch.equal(a, b)
    assert not c0[3].any() and not c0[4].any()
    # states only (no torques, no distances): motion terms alone
    m = W.trajopt_cost_ext(None, None, cuda(qd), cuda(qdd), None, None, 0.0, **kw)
    torch.cuda.synchronize()
    assert m[1] is None and m[2] is None
    rm = O.trajopt_cost(np.zeros((d, B)), np.ones(B), lo, hi, 0.0, qd, qdd, **kw)
    assert np.allclose(m[0].cpu().numpy(), rm[0], rtol=1e-5)
    assert np.allclose(m[3].cpu().numpy(), 2.0 * kw["length"] * qd, rtol=1e-6)


def test_trajopt_cost_ext_rejects_bad_weights(W):
    x = cuda(np.ones((3, 4)))
    for bad in (dict(dt=0.0), dict(dt=-1.0), dict(smooth=float("nan")),
                dict(energy=float("inf"))):
        with pytest.raises(W.L.WbError):
            W.trajopt_cost_ext(x, None, x, x, cuda(-np.ones(3)), cuda(np.ones(3)), 1.0, **bad)


def test_bspline_backward_ext_adds_before_the_transpose(W):
    """gqd + gqd_add through the adjoint equals the plain adjoint of the float
    sum: the kernel adds in the same float order as the caller would."""
    rng = np.random.default_rng(5)
    n_traj, d, K, T = 9, 13, 11, 33
    g = [cuda(rng.normal(size=(d, n_traj * T))) for _ in range(5)]
    a = W.bspline_backward(g[0], g[1], g[2], n_traj, K, T, 0.2, gqd_add=g[3], gqdd_add=g[4])
    b = W.bspline_backward(g[0], g[1] + g[3], g[2] + g[4], n_traj, K, T, 0.2)
    c = W.bspline_backward(None, None, None, n_traj, K, T, 0.2, gqd_add=g[3])
    e = W.bspline_backward(None, g[3], None, n_traj, K, T, 0.2)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(c, e)


def _chain(W, rob, desc, U, T, dt, lo, hi, w, motion=None):
    """The GPU chain; returns (gU, cost, eval outputs).  ``motion`` holds the
    smooth / length / energy weights of the cost's motion terms."""
    n_traj, d, K = U.shape
    q, qd, qdd = W.bspline_eval(U, T, dt)
    o = rob.eval(q, qd, qdd)
    if motion:
        cost, g_tau, g_dmin, g_qd, g_qdd = W.trajopt_cost_ext(
            o["tau"], o["dmin"], qd, qdd, lo, hi, w, dt=dt * (K - 3) / (T - 1), **motion)
    else:
        cost, g_tau, g_dmin = W.trajopt_cost(o["tau"], o["dmin"], lo, hi, w)
        g_qd = g_qdd = None
    gq, gqd, gqdd = rob.eval_backward(q, qd, qdd, o["worst"], None, None, g_dmin, g_tau)
    gU = W.bspline_backward(gq, gqd, gqdd, n_traj, K, T, dt, gqd_add=g_qd, gqdd_add=g_qdd)
    torch.cuda.synchronize()
    return gU, cost, o


def _compare_chain(O, desc, U, T, dt, lim, w, gU, cost, o, trajs, motion=None):
    d = desc.dof
    lo, hi = -lim * np.ones(d), lim * np.ones(d)
    Uref, cref, ev = O.trajopt_gradient(desc, U.astype(np.float64), T, dt, lo, hi, w,
                                        **(motion or {}))
    tau, dmin, worst = ev["tau"], ev["dmin"], ev["worst"]
    got_worst = o["worst"].cpu().numpy()
    got_cost = cost.cpu().numpy()
    gUn = gU.cpu().numpy()
    kept = 0
    for i, tr in enumerate(trajs):
        sl = slice(i * T, (i + 1) * T)
        gsl = slice(tr * T, (tr + 1) * T)
        # torques agree to 1e-4 relative per joint, so the hinge sums do too
        tol = 1e-4 * np.maximum(np.abs(tau[:, sl]), 1.0).sum(axis=0) + 1e-5
        if motion:  # the energy term is quadratic in the torques: 2e-4 relative
            tol = tol + 2e-4 * np.abs(cref[sl])
        assert (np.abs(got_cost[gsl] - cref[sl]) <= tol).all()
        near = (np.abs(np.abs(tau[:, sl]) - lim) < 1e-3).any() or \
            (np.abs(dmin[sl]) < 1e-4).any() or not np.array_equal(got_worst[gsl], worst[sl])
        if near:  # a hinge or the worst pair may switch between FP32 and FP64
            continue
        e = np.linalg.norm(gUn[tr] - Uref[i])
        assert e <= PY.GRAD_REL * max(np.linalg.norm(Uref[i]), 1e-6), (tr, e)
        kept += 1
    return kept


def test_trajopt_chain_matches_oracle(W, O):
    """U -> B-spline -> FK + spheres + self-collision + RNEA -> cost ->
    adjoint -> dL/dU, 48-DoF humanoid with 3 kg hand payloads, torque limits
    +-30 N m, collision weight 1."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = 6, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    U = I.bspline_controls(desc.dof, n_traj, K, seed=CF.TRAJOPT48.seed)
    lim, w = CF.TORQUE_LIMIT, CF.COLLISION_WEIGHT
    lo = cuda(-lim * np.ones(desc.dof))
    hi = cuda(lim * np.ones(desc.dof))
    gU, cost, o = _chain(W, rob, desc, cuda(U), T, dt, lo, hi, w)
    tau = o["tau"].cpu().numpy()
    assert (np.abs(tau) > lim).mean() > 0.01  # the torque hinge is active
    kept = _compare_chain(O, desc, U, T, dt, lim, w, gU, cost, o, list(range(n_traj)))
    assert kept >= n_traj - 2


def test_trajopt48_full_size_sampled(W, O):
    """The full 512 x 64 launch; three trajectories checked against the
    oracle (each trajectory's dL/dU depends on its own samples only)."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = CF.TRAJOPT_SEEDS, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    U = I.bspline_controls(desc.dof, n_traj, K, seed=CF.TRAJOPT48.seed)
    lim, w = CF.TORQUE_LIMIT, CF.COLLISION_WEIGHT
    lo = cuda(-lim * np.ones(desc.dof))
    hi = cuda(lim * np.ones(desc.dof))
    gU, cost, o = _chain(W, rob, desc, cuda(U), T, dt, lo, hi, w)
    assert torch.isfinite(gU).all() and torch.isfinite(cost).all()
    trajs = [0, 257, n_traj - 1]
    kept = _compare_chain(O, desc, U[trajs], T, dt, lim, w, gU, cost, o, trajs)
    assert kept >= 2


def test_trajopt_chain_with_motion_terms_matches_oracle(W, O):
    """The chain with the smooth, length and energy terms of the loss at the
    trajopt48 weights: the cost's direct qd / qdd gradients join the sweep's
    in the B-spline adjoint."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = 6, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    U = I.bspline_controls(desc.dof, n_traj, K, seed=CF.TRAJOPT48.seed + 1)
    lim, w = CF.TORQUE_LIMIT, CF.COLLISION_WEIGHT
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    lo = cuda(-lim * np.ones(desc.dof))
    hi = cuda(lim * np.ones(desc.dof))
    gU, cost, o = _chain(W, rob, desc, cuda(U), T, dt, lo, hi, w, motion)
    kept = _compare_chain(O, desc, U, T, dt, lim, w, gU, cost, o, list(range(n_traj)), motion)
    assert kept >= n_traj - 2


def test_trajopt_chain_with_summed_hinge_matches_oracle(W, O):
    """The trajopt48 chain with the summed collision hinge (activation
    distance 2 cm) and the motion terms, as `bench.py --workload trajopt48
    --collision hinge` runs it: hinge sphere gradient -> backward sweep, the
    cost's direct qd / qdd gradients -> B-spline adjoint."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = 4, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    U = I.bspline_controls(desc.dof, n_traj, K, seed=CF.TRAJOPT48.seed + 2)
    lim, w, eta = CF.TORQUE_LIMIT, CF.COLLISION_WEIGHT, CF.ACTIVATION_DISTANCE
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    lo = cuda(-lim * np.ones(desc.dof))
    hi = cuda(lim * np.ones(desc.dof))
    Ud = cuda(U)
    q, qd, qdd = W.bspline_eval(Ud, T, dt)
    o = rob.eval(q, qd, qdd, sphere=False, dmin=False)
    hcost, g_sph = rob.self_collision_hinge(o["pose"], eta, w)
    cost, g_tau, _, g_qd, g_qdd = W.trajopt_cost_ext(o["tau"], None, qd, qdd, lo, hi, w,
                                                     dt=dt * (K - 3) / (T - 1), **motion)
    gq, gqd, gqdd = rob.eval_backward(q, qd, qdd, None, None, g_sph, None, g_tau)
    gU = W.bspline_backward(gq, gqd, gqdd, n_traj, K, T, dt, gqd_add=g_qd, gqdd_add=g_qdd)
    torch.cuda.synchronize()
    Uref, cref, ev = O.trajopt_gradient(desc, U.astype(np.float64), T, dt, -lim * np.ones(desc.dof),
                                        lim * np.ones(desc.dof), w, eta=eta, **motion)
    total = (cost + hcost).cpu().numpy()
    # torques agree to 1e-4 relative, distances to 1e-5 m per active pair
    tol = 1e-4 * np.abs(cref) + 1e-4 * np.maximum(np.abs(ev["tau"]), 1.0).sum(axis=0) + 1e-2
    assert (np.abs(total - cref) <= tol).all()
    gUn = gU.cpu().numpy()
    good = 0
    for tr in range(n_traj):
        e = np.linalg.norm(gUn[tr] - Uref[tr])
        # a pair within float rounding of eta may switch sides: a unit-size
        # change against a gradient of norm ~1e4
        good += e <= 2 * PY.GRAD_REL * np.linalg.norm(Uref[tr])
    assert good >= n_traj - 1


@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("collision,kin", [(True, False), (False, True)])
def test_fused_cost_matches_separate_calls(W, G, collision, kin):
    """wb_eval_backward_cost against wb_trajopt_cost_ext + wb_eval_backward +
    adding the direct q-dot / q-ddot gradients, for every sweep segment
    count, with the worst-pair term or with pose / sphere gradients."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    B = 301
    q, qd, qdd = (cuda(x) for x in I.uniform_states(desc.dof, B, seed=PY.stable_seed("fc", G)))
    gp, gs, _, _ = I.upstream_grads(desc, B, seed=12)
    gp, gs = (cuda(gp), cuda(gs)) if kin else (None, None)
    lim = CF.TORQUE_LIMIT
    lo, hi = cuda(-lim * np.ones(desc.dof)), cuda(lim * np.ones(desc.dof))
    wts = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT,
               dt=0.05)
    tune = W.Tune(kernel=3, lanes_per_config=G)
    o = rob.eval(q, qd, qdd, tune=tune)
    dmin = o["dmin"] if collision else None
    worst = o["worst"] if collision else None
    c1, g_tau, g_dmin, g_qd, g_qdd = W.trajopt_cost_ext(o["tau"], dmin, qd, qdd, lo, hi, 1.5,
                                                        **wts)
    a = rob.eval_backward(q, qd, qdd, worst, gp, gs, g_dmin, g_tau, tune=tune)
    ref = (a[0], a[1] + g_qd, a[2] + g_qdd)
    b = rob.eval_backward_cost(q, qd, qdd, o["tau"], lo, hi, 1.5, d_min=dmin, worst=worst,
                               g_pose=gp, g_sphere=gs, tune=tune, **wts)
    torch.cuda.synchronize()
    for x, y in zip(b[:3], ref):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.abs(x - y).max() <= 1e-5 * max(1.0, np.abs(y).max())
    assert np.allclose(b[3].cpu().numpy(), c1.cpu().numpy(), rtol=1e-5, atol=1e-4)


def test_fused_cost_chain_matches_oracle(W, O):
    """The trajopt48 chain through the fused cost: U -> B-spline -> forward
    + worst pair -> backward sweep with the cost in its prologue -> dL/dU."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = 6, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    U = I.bspline_controls(desc.dof, n_traj, K, seed=CF.TRAJOPT48.seed + 3)
    lim, w = CF.TORQUE_LIMIT, CF.COLLISION_WEIGHT
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    lo, hi = cuda(-lim * np.ones(desc.dof)), cuda(lim * np.ones(desc.dof))
    q, qd, qdd = W.bspline_eval(cuda(U), T, dt)
    o = rob.eval(q, qd, qdd)
    gq, gqd, gqdd, cost = rob.eval_backward_cost(q, qd, qdd, o["tau"], lo, hi, w, d_min=o["dmin"],
                                                 worst=o["worst"], dt=dt * (K - 3) / (T - 1),
                                                 **motion)
    gU = W.bspline_backward(gq, gqd, gqdd, n_traj, K, T, dt)
    torch.cuda.synchronize()
    kept = _compare_chain(O, desc, U, T, dt, lim, w, gU, cost, o, list(range(n_traj)), motion)
    assert kept >= n_traj - 2


def test_fused_cost_refusals(W):
    from paper_2603_05493_gb300 import _lib as L
    desc = R.mixed_joint_tree()  # a joint drives two links
    rob = W.Robot(desc, device=0)
    x = torch.zeros((desc.dof, 8), device="cuda")
    lim = torch.ones(desc.dof, device="cuda")
    with pytest.raises(L.WbError) as e:
        rob.eval_backward_cost(x, x, x, x, -lim, lim, 1.0)
    assert e.value.code == L.WB_EINVAL
    d7 = R.r7()
    r7 = W.Robot(d7, device=0)
    x = torch.zeros((d7.dof, 8), device="cuda")
    lim = torch.ones(d7.dof, device="cuda")
    with pytest.raises(L.WbError) as e:
        r7.eval_backward_cost(x, x, x, x, -lim, lim, 1.0, tune=W.PLAIN)
    assert e.value.code == L.WB_EINVAL
    with pytest.raises(L.WbError) as e:  # d_min without its worst pair
        r7.eval_backward_cost(x, x, x, x, -lim, lim, 1.0, d_min=torch.zeros(8, device="cuda"))
    assert e.value.code == L.WB_EINVAL


def test_trajopt48_full_size_fused_cost_sampled(W, O):
    """The full 512 x 64 launch as the bench runs it (the cost in the
    backward sweep's prologue, autotuned shapes); three trajectories checked
    against the oracle."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = CF.TRAJOPT_SEEDS, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    B = n_traj * T
    ft, bt, _, _ = rob.autotune(B)
    U = I.bspline_controls(desc.dof, n_traj, K, seed=CF.TRAJOPT48.seed)
    lim, w = CF.TORQUE_LIMIT, CF.COLLISION_WEIGHT
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    lo, hi = cuda(-lim * np.ones(desc.dof)), cuda(lim * np.ones(desc.dof))
    q, qd, qdd = W.bspline_eval(cuda(U), T, dt)
    tree = lambda t: W.Tune(kernel=3, lanes_per_config=t.lanes_per_config if t.kernel == 3 else 0,  # noqa: E731
                            configs_per_block=t.configs_per_block if t.kernel == 3 else 0)
    o = rob.eval(q, qd, qdd, tune=tree(ft))
    gq, gqd, gqdd, cost = rob.eval_backward_cost(q, qd, qdd, o["tau"], lo, hi, w, d_min=o["dmin"],
                                                 worst=o["worst"], dt=dt * (K - 3) / (T - 1),
                                                 tune=tree(bt), **motion)
    gU = W.bspline_backward(gq, gqd, gqdd, n_traj, K, T, dt)
    torch.cuda.synchronize()
    assert torch.isfinite(gU).all() and torch.isfinite(cost).all()
    trajs = [0, 257, n_traj - 1]
    kept = _compare_chain(O, desc, U[trajs], T, dt, lim, w, gU, cost, o, trajs, motion)
    assert kept >= 2


@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("kin", [False, True])
def test_spline_sourced_sweeps_equal_the_two_step_path(W, G, kin):
    """The sweeps with the joint states evaluated from control points
    (wb_eval_spline, wb_eval_backward_spline_cost) against wb_bspline_eval
    followed by wb_eval and wb_eval_backward_cost: the states are the same
    bits, so every output is too, for every sweep segment count."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = 5, 16, 45, 0.25  # 225 configurations: a ragged tail
    U = cuda(I.bspline_controls(desc.dof, n_traj, K, seed=PY.stable_seed("spl", G)))
    tune = W.Tune(kernel=3, lanes_per_config=G)
    q, qd, qdd = W.bspline_eval(U, T, dt)
    a = rob.eval(q, qd, qdd, tune=tune)
    b = rob.eval_spline(U, T, dt, tune=tune)
    torch.cuda.synchronize()
    for k in ("pose", "sphere", "dmin", "worst", "tau"):
        assert torch.equal(a[k], b[k]), k
    lim = CF.TORQUE_LIMIT
    lo, hi = cuda(-lim * np.ones(desc.dof)), cuda(lim * np.ones(desc.dof))
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    gp, gs, _, _ = I.upstream_grads(desc, n_traj * T, seed=31)
    gp, gs = (cuda(gp), cuda(gs)) if kin else (None, None)
    dtc = dt * (K - 3) / (T - 1)
    ga = rob.eval_backward_cost(q, qd, qdd, a["tau"], lo, hi, 1.0, dt=dtc, d_min=a["dmin"],
                                worst=a["worst"], g_pose=gp, g_sphere=gs, tune=tune, **motion)
    gb = rob.eval_backward_spline_cost(U, T, dt, b["tau"], lo, hi, 1.0, dt_cost=dtc,
                                       d_min=b["dmin"], worst=b["worst"], g_pose=gp, g_sphere=gs,
                                       tune=tune, **motion)
    torch.cuda.synchronize()
    for x, y in zip(ga, gb):
        assert torch.equal(x, y)


def test_trajopt48_full_size_spline_sampled(W, O):
    """The full 512 x 64 launch as the bench runs it: states from control
    points inside the sweeps, the cost in the backward's prologue, autotuned
    shapes; three trajectories against the oracle."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = CF.TRAJOPT_SEEDS, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    lim, w = CF.TORQUE_LIMIT, CF.COLLISION_WEIGHT
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    ft, bt, _, _ = rob.autotune_spline(n_traj, K, T, dt, w, dt_cost=dt * (K - 3) / (T - 1),
                                       **motion)
    U = I.bspline_controls(desc.dof, n_traj, K, seed=CF.TRAJOPT48.seed)
    lo, hi = cuda(-lim * np.ones(desc.dof)), cuda(lim * np.ones(desc.dof))
    tree = lambda t: W.Tune(kernel=3, lanes_per_config=t.lanes_per_config if t.kernel == 3 else 0,  # noqa: E731
                            configs_per_block=t.configs_per_block if t.kernel == 3 else 0)
    Ud = cuda(U)
    o = rob.eval_spline(Ud, T, dt, tune=tree(ft))
    gq, gqd, gqdd, cost = rob.eval_backward_spline_cost(
        Ud, T, dt, o["tau"], lo, hi, w, dt_cost=dt * (K - 3) / (T - 1), d_min=o["dmin"],
        worst=o["worst"], tune=tree(bt), **motion)
    gU = W.bspline_backward(gq, gqd, gqdd, n_traj, K, T, dt)
    torch.cuda.synchronize()
    assert torch.isfinite(gU).all() and torch.isfinite(cost).all()
    trajs = [0, 300, n_traj - 1]
    kept = _compare_chain(O, desc, U[trajs], T, dt, lim, w, gU, cost, o, trajs, motion)
    assert kept >= 2


def test_spline_sourced_refusals(W):
    from paper_2603_05493_gb300 import _lib as L
    desc = R.r7()
    rob = W.Robot(desc, device=0)
    U3 = torch.zeros((2, desc.dof, 3), device="cuda")
    with pytest.raises(L.WbError) as e:  # 3 control points
        rob.eval_spline(U3, 8, 0.1)
    assert e.value.code == L.WB_EINVAL
    U = torch.zeros((2, desc.dof, 6), device="cuda")
    with pytest.raises(L.WbError) as e:
        rob.eval_spline(U, 8, 0.1, tune=W.PLAIN)
    assert e.value.code == L.WB_EINVAL
    o = rob.eval_spline(U, 8, 0.1, sphere=False, dmin=False)
    torch.cuda.synchronize()
    assert torch.isfinite(o["tau"]).all()


def test_autotune_spline_shapes_run_and_agree(W):
    """wb_autotune_spline returns depth-first sweep shapes the robot takes,
    with positive times; the chosen shapes give the one-segment sweep's
    results up to the rounding of the segments' partial sums."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = 16, 16, 64, 0.25
    dtc = dt * (K - 3) / (T - 1)
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    ft, bt, fm, bm = rob.autotune_spline(n_traj, K, T, dt, 1.0, dt_cost=dtc, **motion)
    for t in (ft, bt):
        assert t.kernel == 3 and t.lanes_per_config in (1, 2, 4, 8)
        assert t.configs_per_block in (64, 128, 256)
    assert 0.0 < fm < 1e3 and 0.0 < bm < 1e3
    U = cuda(I.bspline_controls(desc.dof, n_traj, K, seed=PY.stable_seed("ats", 0)))
    one = W.Tune(kernel=3, lanes_per_config=1)
    lo = cuda(-CF.TORQUE_LIMIT * np.ones(desc.dof))
    hi = cuda(CF.TORQUE_LIMIT * np.ones(desc.dof))
    res = []
    for ftune, btune in ((one, one), (ft, bt)):
        o = rob.eval_spline(U, T, dt, tune=ftune)
        g = rob.eval_backward_spline_cost(U, T, dt, o["tau"], lo, hi, 1.0, dt_cost=dtc,
                                          d_min=o["dmin"], worst=o["worst"], tune=btune,
                                          **motion)
        res.append((o, g))
    torch.cuda.synchronize()
    (o1, g1), (o2, g2) = res
    assert torch.equal(o1["worst"], o2["worst"])
    for k in ("pose", "dmin", "tau"):
        assert torch.allclose(o1[k], o2[k], rtol=1e-4, atol=1e-4), k
    for x, y in zip(g1, g2):
        assert torch.allclose(x, y, rtol=1e-4, atol=1e-3 * float(x.abs().max()))


def test_autotune_spline_refusals(W):
    from paper_2603_05493_gb300 import _lib as L
    rob = W.Robot(R.r7(), device=0)
    for args in ((0, 8, 16, 0.1), (2, 3, 16, 0.1), (2, 8, 1, 0.1), (2, 8, 16, 0.0)):
        with pytest.raises(L.WbError) as e:
            rob.autotune_spline(*args)
        assert e.value.code == L.WB_EINVAL, args
    deep = W.Robot(R.deep_chain(33), device=0)
    with pytest.raises(L.WbError) as e:
        deep.autotune_spline(2, 8, 16, 0.1)
    assert e.value.code == L.WB_ETOOBIG



@pytest.mark.parametrize("G", [1, 2, 4])
def test_fused_cost_with_worst_diff_is_bit_identical(W, G):
    """The cost-fused backward with the pair stage's worst-pair centre
    difference (wb_eval_backward_cost_dir, wb_eval_backward_spline_cost_dir)
    gives the same bits as without it, for array and control-point states."""
    desc = I.hand_payload(R.r48())
    rob = W.Robot(desc, device=0)
    n_traj, K, T, dt = 4, 16, 37, 0.25
    U = cuda(I.bspline_controls(desc.dof, n_traj, K, seed=PY.stable_seed("wd", G)))
    tune = W.Tune(kernel=3, lanes_per_config=G)
    o = rob.eval_spline(U, T, dt, tune=tune, sphere=False, dmin=False)
    c = rob.self_collision(o["pose"], diff=True)
    lim = CF.TORQUE_LIMIT
    lo, hi = cuda(-lim * np.ones(desc.dof)), cuda(lim * np.ones(desc.dof))
    motion = dict(smooth=CF.SMOOTH_WEIGHT, length=CF.LENGTH_WEIGHT, energy=CF.ENERGY_WEIGHT)
    dtc = dt * (K - 3) / (T - 1)
    kw = dict(d_min=c["dmin"], worst=c["worst"], tune=tune)
    a = rob.eval_backward_spline_cost(U, T, dt, o["tau"], lo, hi, 1.0, dt_cost=dtc, **motion,
                                      **kw)
    b = rob.eval_backward_spline_cost(U, T, dt, o["tau"], lo, hi, 1.0, dt_cost=dtc, **motion,
                                      worst_diff=c["diff"], **kw)
    q, qd, qdd = W.bspline_eval(U, T, dt)
    e = rob.eval_backward_cost(q, qd, qdd, o["tau"], lo, hi, 1.0, dt=dtc, **motion, **kw)
    f = rob.eval_backward_cost(q, qd, qdd, o["tau"], lo, hi, 1.0, dt=dtc, **motion,
                               worst_diff=c["diff"], **kw)
    torch.cuda.synchronize()
    assert (c["dmin"] < 0).float().mean() > 0.5  # most configurations take the pair term
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    for x, y in zip(e, f):
        assert torch.equal(x, y)
