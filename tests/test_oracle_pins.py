"""Pins of the FP64 oracle to things other than itself: closed forms,
invariants, an independent Lagrangian formulation, library routines and finite
differences.  CPU only."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

from synthetic import robots as R
from synthetic import inputs as I


def states(robot, B, seed):
    return I.uniform_states(robot.dof, B, seed)


def ev(O, robot, q, qd=None, qdd=None, **kw):
    return O.evaluate(robot, np.asarray(q, float).reshape(robot.dof, -1),
                      None if qd is None else np.asarray(qd, float).reshape(robot.dof, -1),
                      None if qdd is None else np.asarray(qdd, float).reshape(robot.dof, -1),
                      nthreads=1, **kw)


def tau_of(O, robot, q, qd, qdd):
    return ev(O, robot, q, qd, qdd, want=("tau",))["tau"][:, 0]


# ---------------------------------------------------------------------------
# forward kinematics
# ---------------------------------------------------------------------------

def test_planar_2link_closed_form(oracle_lib):
    """Sec. 6.1.1 FK on the 2-link planar arm: x = l1 cos q1 + l2 cos(q1+q2),
    y = l1 sin q1 + l2 sin(q1+q2), z = 0."""
    O = oracle_lib
    l1, l2 = 0.5, 0.25
    rob = R.planar_2link(l1, l2)
    rng = np.random.default_rng(0)
    for _ in range(20):
        q1, q2 = rng.uniform(-np.pi, np.pi, 2)
        o = ev(O, rob, [q1, q2])
        tip = o["sph"][0, 1]
        assert np.allclose(tip, [l1 * np.cos(q1) + l2 * np.cos(q1 + q2),
                                 l1 * np.sin(q1) + l2 * np.sin(q1 + q2), 0.0], atol=1e-14)
        p2 = o["pose"][0, 1, 9:]
        assert np.allclose(p2, [l1 * np.cos(q1), l1 * np.sin(q1), 0], atol=1e-14)
        R2 = o["pose"][0, 1, :9].reshape(3, 3)
        c, s = np.cos(q1 + q2), np.sin(q1 + q2)
        assert np.allclose(R2, [[c, -s, 0], [s, c, 0], [0, 0, 1]], atol=1e-14)


def _homog(T12):
    H = np.eye(4)
    H[:3, :3] = np.asarray(T12[:9]).reshape(3, 3)
    H[:3, 3] = T12[9:]
    return H


@pytest.mark.parametrize("mk", [R.r7, R.r48, R.mixed_joint_tree])
def test_zero_config_is_product_of_fixed_transforms(oracle_lib, mk):
    """At q = 0 (and zero mimic offsets) each world pose is the product of the
    fixed transforms along the chain."""
    O = oracle_lib
    rob = mk()
    rob.mimic_off[:] = 0.0
    o = ev(O, rob, np.zeros(rob.dof))
    for k in range(rob.n):
        H = np.eye(4)
        chain = []
        j = k
        while j >= 0:
            chain.append(j)
            j = rob.parent[j]
        for j in reversed(chain):
            H = H @ _homog(rob.T_fixed[j])
        got = _homog(o["pose"][0, k])
        assert np.allclose(got, H, atol=1e-13)


@pytest.mark.parametrize("mk", [R.r7, R.r48, R.mixed_joint_tree])
def test_rotations_orthonormal_and_offsets_preserved(oracle_lib, mk):
    O = oracle_lib
    rob = mk()
    q, _, _ = states(rob, 32, 5)
    o = O.evaluate(rob, q, want=("pose",), nthreads=1)
    Rm = o["pose"][:, :, :9].reshape(-1, rob.n, 3, 3)
    eye = np.einsum("bkji,bkjl->bkil", Rm, Rm)
    # fixed rotations are float32-rounded: the invariant holds up to their own
    # deviation from orthonormality, accumulated along the chain
    Rf = rob.T_fixed[:, :9].reshape(-1, 3, 3)
    dev = np.abs(np.einsum("kji,kjl->kil", Rf, Rf) - np.eye(3)).max()
    tol = 1e-12 + 3 * (rob.depth().max() + 1) * dev
    assert np.abs(eye - np.eye(3)).max() <= tol
    assert np.abs(np.linalg.det(Rm) - 1).max() <= tol
    p = o["pose"][:, :, 9:]
    for k in range(rob.n):
        pa = rob.parent[k]
        if pa >= 0 and rob.jtype[k] == R.REVOLUTE:
            dist = np.linalg.norm(p[:, k] - p[:, pa], axis=1)
            assert np.allclose(dist, np.linalg.norm(rob.T_fixed[k, 9:]), atol=1e-13)


def test_prismatic_moves_along_axis(oracle_lib):
    """A prismatic joint translates its link by q along the joint axis
    (expressed in the parent through the fixed rotation)."""
    O = oracle_lib
    rob = R.mixed_joint_tree()
    k = 1
    assert rob.jtype[k] == R.PRISMATIC
    rng = np.random.default_rng(1)
    q = rng.uniform(-1, 1, rob.dof)
    o0 = ev(O, rob, q)
    q2 = q.copy()
    q2[rob.jidx[k]] += 0.3
    o1 = ev(O, rob, q2)
    Rpa = o0["pose"][0, rob.parent[k], :9].reshape(3, 3)
    Rf = rob.T_fixed[k, :9].reshape(3, 3)
    step = Rpa @ Rf @ (rob.axis[k] / np.linalg.norm(rob.axis[k])) * 0.3
    assert np.allclose(o1["pose"][0, k, 9:] - o0["pose"][0, k, 9:], step, atol=1e-13)


# ---------------------------------------------------------------------------
# spheres and self-collision
# ---------------------------------------------------------------------------

def _slider_robot(radii):
    """Prismatic sliders along x from the world origin, one sphere each: the
    sphere centres are exactly (q_k, 0, 0)."""
    n = len(radii)
    return R._plain("sliders", [-1] * n, [R.PRISMATIC] * n, [[1, 0, 0]] * n,
                    [R._Tp(0, 0, 0)] * n, mass=[1.0] * n, com=np.zeros((n, 3)),
                    Icom=[[0.1, 0.1, 0.1, 0, 0, 0]] * n, sph_link=list(range(n)),
                    sph_c=np.zeros((n, 3)), sph_r=radii,
                    pairs=[[i, j] for i in range(n) for j in range(i + 1, n)])


def test_hand_built_sphere_cases(oracle_lib):
    """Three spheres at known positions: distances |xi-xj| - ri - rj; exactly
    touching spheres (d = 0) are not colliding under the strict test."""
    O = oracle_lib
    rob = _slider_robot([0.25, 0.125, 0.5])
    # sphere 0 at 0, sphere 1 at 0.375 (touching 0), sphere 2 at 2.0
    o = ev(O, rob, [0.0, 0.375, 2.0], want=("dmin", "collide"))
    assert o["dmin"][0] == 0.0 and o["worst"][0] == 0
    assert list(o["collide"][0]) == [0, 0, 0]
    # move sphere 2 to 0.5: pair (1,2) = 0.125 - 0.625 = -0.5, (0,2) = 0.5 - 0.75
    o = ev(O, rob, [0.0, 0.375, 0.5], want=("dmin", "collide"))
    assert o["dmin"][0] == -0.5 and o["worst"][0] == 2
    assert list(o["collide"][0]) == [0, 1, 1]
    # exact tie between pair 0 (0,1) and pair 2 (1,2): the smaller index wins
    o = ev(O, rob, [0.0, 0.375, 1.0], want=("dmin",))
    assert o["dmin"][0] == 0.0 and o["worst"][0] == 0


@pytest.mark.parametrize("mk", [R.r7, R.r23, R.r48])
def test_pairs_match_library_distance_matrix(oracle_lib, mk):
    """d_min / worst / collide against scipy's cdist over the masked pairs."""
    O = oracle_lib
    rob = mk()
    q, _, _ = states(rob, 8, 11)
    o = O.evaluate(rob, q, want=("sph", "dmin", "collide"), nthreads=1)
    i, j = rob.pairs[:, 0], rob.pairs[:, 1]
    for b in range(q.shape[1]):
        D = cdist(o["sph"][b], o["sph"][b])[i, j] - rob.sph_r[i] - rob.sph_r[j]
        assert abs(o["dmin"][b] - D.min()) <= 1e-13
        assert abs(D[o["worst"][b]] - D.min()) <= 1e-13
        assert np.array_equal(o["collide"][b].astype(bool), D < 0)


def test_pair_permutation_invariance(oracle_lib):
    O = oracle_lib
    rob = R.r23()
    q, _, _ = states(rob, 16, 12)
    base = O.evaluate(rob, q, want=("dmin",), nthreads=1)
    perm = np.random.default_rng(3).permutation(rob.P)
    shuf = rob.with_pairs(rob.pairs[perm])
    o = O.evaluate(shuf, q, want=("dmin",), nthreads=1)
    assert np.array_equal(o["dmin"], base["dmin"])
    assert np.array_equal(perm[o["worst"]], base["worst"])


# ---------------------------------------------------------------------------
# inverse dynamics
# ---------------------------------------------------------------------------

def test_single_pendulum_closed_form(oracle_lib):
    """tau = (Ixx + m l^2) qdd + m g l cos q, velocity terms exactly 0."""
    O = oracle_lib
    rob = R.pendulum(2.0, 0.75, 0.05)
    # the parameters as stored (float32-representable values)
    m, l, Ixx, g = rob.mass[0], rob.com[0, 1], rob.Icom[0, 0], -rob.gravity[2]
    rng = np.random.default_rng(2)
    for _ in range(20):
        q, qd, qdd = rng.uniform(-3, 3, 3)
        t = tau_of(O, rob, [q], [qd], [qdd])[0]
        ref = (Ixx + m * l * l) * qdd + m * g * l * np.cos(q)
        assert abs(t - ref) <= 1e-12 * max(1.0, abs(ref))
        assert abs(tau_of(O, rob, [q], [qd], [0.0])[0] - tau_of(O, rob, [q], [0.0], [0.0])[0]) \
            <= 1e-12


def _world_com(rob, pose):
    """World CoM of every link from the oracle's poses [n][12]."""
    Rm = pose[:, :9].reshape(-1, 3, 3)
    return np.einsum("kij,kj->ki", Rm, rob.com) + pose[:, 9:]


def _potential(O, rob, q):
    pose = ev(O, rob, q, want=("pose",))["pose"][0]
    c = _world_com(rob, pose)
    V = -np.sum(rob.mass[:, None] * c * rob.gravity[None, :])
    if len(rob.pm_link):
        Rm = pose[:, :9].reshape(-1, 3, 3)
        x = np.einsum("kij,kj->ki", Rm[rob.pm_link], rob.pm_pos) + pose[rob.pm_link, 9:]
        V -= np.sum(rob.pm_mass[:, None] * x * rob.gravity[None, :])
    return V


@pytest.mark.parametrize("mk", [R.r7, R.mixed_joint_tree, R.r23,
                                lambda: I.hand_payload(R.r48())])
def test_gravity_torque_is_potential_gradient(oracle_lib, mk):
    """tau(q, 0, 0) = dV/dq, V = -sum m g.c(q), by central differences."""
    O = oracle_lib
    rob = mk()
    q, _, _ = states(rob, 2, 21)
    h = 1e-6
    for b in range(2):
        qb = q[:, b].astype(float)
        tg = tau_of(O, rob, qb, np.zeros(rob.dof), np.zeros(rob.dof))
        fd = np.zeros(rob.dof)
        for j in range(rob.dof):
            e = np.zeros(rob.dof)
            e[j] = h
            fd[j] = (_potential(O, rob, qb + e) - _potential(O, rob, qb - e)) / (2 * h)
        assert np.abs(tg - fd).max() <= 1e-7 * max(1.0, np.abs(tg).max())


def test_axes_parallel_to_gravity_have_no_static_torque(oracle_lib):
    O = oracle_lib
    rob = R.chain_along_gravity()
    q, _, _ = states(rob, 4, 8)
    o = O.evaluate(rob, q, np.zeros_like(q), np.zeros_like(q), want=("tau",), nthreads=1)
    assert np.abs(o["tau"]).max() <= 1e-12


def _jacobian_mass_matrix(O, rob, q, h=1e-6):
    """M(q) = sum_k m_k Jv^T Jv + Jw^T (R Ic R^T) Jw from geometric Jacobians,
    the Jacobians taken by central differences of forward kinematics alone."""
    d = rob.dof

    def kin(qq):
        pose = ev(O, rob, qq, want=("pose",))["pose"][0]
        return pose[:, :9].reshape(-1, 3, 3), _world_com(rob, pose), pose

    R0, c0, pose0 = kin(q)
    Jv = np.zeros((rob.n, 3, d))
    Jw = np.zeros((rob.n, 3, d))
    Jp = np.zeros((len(rob.pm_link), 3, d))
    for j in range(d):
        e = np.zeros(d)
        e[j] = h
        Rp, cp, pp = kin(q + e)
        Rm_, cm, pm = kin(q - e)
        Jv[:, :, j] = (cp - cm) / (2 * h)
        dR = (Rp - Rm_) / (2 * h)
        W = np.einsum("kij,klj->kil", dR, R0)   # dR R^T = [w]^
        Jw[:, :, j] = np.stack([W[:, 2, 1], W[:, 0, 2], W[:, 1, 0]], axis=1)
        for m, l in enumerate(rob.pm_link):
            xp = pp[l, :9].reshape(3, 3) @ rob.pm_pos[m] + pp[l, 9:]
            xm = pm[l, :9].reshape(3, 3) @ rob.pm_pos[m] + pm[l, 9:]
            Jp[m, :, j] = (xp - xm) / (2 * h)
    M = np.zeros((d, d))
    for k in range(rob.n):
        ic = rob.Icom[k]
        Ic = np.array([[ic[0], ic[3], ic[4]], [ic[3], ic[1], ic[5]], [ic[4], ic[5], ic[2]]])
        Iw = R0[k] @ Ic @ R0[k].T
        M += rob.mass[k] * Jv[k].T @ Jv[k] + Jw[k].T @ Iw @ Jw[k]
    for m in range(len(rob.pm_link)):
        M += rob.pm_mass[m] * Jp[m].T @ Jp[m]
    return M


def _rnea_mass_matrix(O, rob, q):
    d = rob.dof
    z = np.zeros(d)
    t0 = tau_of(O, rob, q, z, z)
    return np.stack([tau_of(O, rob, q, z, np.eye(d)[j]) - t0 for j in range(d)], axis=1)


@pytest.mark.parametrize("mk", [R.r7, R.mixed_joint_tree, R.r23,
                                lambda: I.hand_payload(R.r48())])
def test_lagrangian_mass_matrix(oracle_lib, mk):
    """tau(q,0,qdd) - tau(q,0,0) = M(q) qdd with M from geometric Jacobians;
    M symmetric positive definite."""
    O = oracle_lib
    rob = mk()
    q, _, _ = states(rob, 1, 31)
    q = q[:, 0].astype(float)
    Mj = _jacobian_mass_matrix(O, rob, q)
    Mr = _rnea_mass_matrix(O, rob, q)
    scale = np.abs(Mj).max()
    assert np.abs(Mr - Mj).max() <= 1e-7 * scale
    assert np.abs(Mr - Mr.T).max() <= 1e-12 * scale
    assert np.linalg.eigvalsh(0.5 * (Mr + Mr.T)).min() > 0


@pytest.mark.parametrize("mk", [R.r7, R.mixed_joint_tree])
def test_coriolis_from_christoffel_symbols(oracle_lib, mk):
    """tau(q,qd,0) - tau(q,0,0) = sum_jk Gamma_ijk qd_j qd_k with Gamma from
    central differences of M(q)."""
    O = oracle_lib
    rob = mk()
    q, qd, _ = states(rob, 1, 41)
    q = q[:, 0].astype(float)
    qd = qd[:, 0].astype(float)
    d = rob.dof
    h = 1e-5
    dM = np.zeros((d, d, d))  # dM[i, j, k] = dM_ij / dq_k
    for k in range(d):
        e = np.zeros(d)
        e[k] = h
        dM[:, :, k] = (_rnea_mass_matrix(O, rob, q + e) - _rnea_mass_matrix(O, rob, q - e)) / (2 * h)
    G = 0.5 * (dM + dM.transpose(0, 2, 1) - dM.transpose(2, 0, 1))  # [i,j,k]: dM_jk/dq_i last
    c = np.einsum("ijk,j,k->i", G, qd, qd)
    z = np.zeros(d)
    got = tau_of(O, rob, q, qd, z) - tau_of(O, rob, q, z, z)
    assert np.abs(got - c).max() <= 1e-6 * max(1.0, np.abs(c).max())


def test_power_balance_along_smooth_trajectory(oracle_lib):
    """qd^T (tau - g(q)) = d/dt (1/2 qd^T M qd) along q(t) = a + b t + c t^2."""
    O = oracle_lib
    rob = R.mixed_joint_tree()
    d = rob.dof
    rng = np.random.default_rng(5)
    a, b, c = rng.uniform(-1, 1, (3, d))

    def state(t):
        return a + b * t + c * t * t, b + 2 * c * t, 2 * c

    def kinetic(t):
        qq, vv, _ = state(t)
        return 0.5 * vv @ _rnea_mass_matrix(O, rob, qq) @ vv

    t0, h = 0.3, 1e-5
    qq, vv, aa = state(t0)
    z = np.zeros(d)
    power = vv @ (tau_of(O, rob, qq, vv, aa) - tau_of(O, rob, qq, z, z))
    dK = (kinetic(t0 + h) - kinetic(t0 - h)) / (2 * h)
    assert abs(power - dK) <= 1e-7 * max(1.0, abs(power))


def test_tau_affine_in_qdd(oracle_lib):
    O = oracle_lib
    rob = R.r48()
    q, qd, qdd = states(rob, 3, 51)
    q, qd = q[:, 0].astype(float), qd[:, 0].astype(float)
    a1, a2 = qdd[:, 1].astype(float), qdd[:, 2].astype(float)
    z = np.zeros(rob.dof)
    lhs = tau_of(O, rob, q, qd, a1 + a2) - tau_of(O, rob, q, qd, a1)
    rhs = tau_of(O, rob, q, qd, a2) - tau_of(O, rob, q, qd, z)
    assert np.abs(lhs - rhs).max() <= 1e-10 * max(1.0, np.abs(lhs).max())


def test_point_payload_adds_its_gravity_torque(oracle_lib):
    """A point mass m at x on a link adds m (w_j x (x - o_j)) . (-g) to the
    static torque of every ancestor joint j."""
    O = oracle_lib
    base = R.r48()
    loaded = I.hand_payload(base)
    q, _, _ = states(base, 2, 61)
    z = np.zeros(base.dof)
    for b in range(2):
        qb = q[:, b].astype(float)
        dt = tau_of(O, loaded, qb, z, z) - tau_of(O, base, qb, z, z)
        pose = ev(O, base, qb, want=("pose",))["pose"][0]
        ref = np.zeros(base.dof)
        for l, m, pp in zip(loaded.pm_link, loaded.pm_mass, loaded.pm_pos):
            x = pose[l, :9].reshape(3, 3) @ pp + pose[l, 9:]
            k = l
            while k >= 0:
                if base.jtype[k] == R.REVOLUTE:
                    w = pose[k, :9].reshape(3, 3) @ (base.axis[k] / np.linalg.norm(base.axis[k]))
                    ref[base.jidx[k]] += m * np.cross(w, x - pose[k, 9:]) @ (-base.gravity)
                k = base.parent[k]
        assert np.abs(dt - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------

def _loss(O, rob, q, qd, qdd, gp, gs, gm, gt):
    o = O.evaluate(rob, q[:, None], qd[:, None], qdd[:, None], nthreads=1)
    return (np.sum(gp * o["pose"][0]) + np.sum(gs * o["sph"][0]) + gm * o["dmin"][0]
            + np.sum(gt * o["tau"][:, 0]))


@pytest.mark.parametrize("mk", [R.r7, R.mixed_joint_tree, R.r23])
def test_dual_gradient_matches_central_differences(oracle_lib, mk):
    O = oracle_lib
    rob = mk()
    B = 2
    q, qd, qdd = states(rob, B, 71)
    gp, gs, gm, gt = I.upstream_grads(rob, B, 72)
    gq, gqd, gqdd = O.gradient(rob, q, qd, qdd, gp, gs, gm, gt, nthreads=1)
    h = 1e-6
    for b in range(B):
        args = [x[:, b].astype(float) for x in (q, qd, qdd)]
        ups = (gp[b].astype(float), gs[b].astype(float), float(gm[b]), gt[:, b].astype(float))
        for which, g in enumerate((gq, gqd, gqdd)):
            fd = np.zeros(rob.dof)
            for j in range(rob.dof):
                ap = [a.copy() for a in args]
                am = [a.copy() for a in args]
                ap[which][j] += h
                am[which][j] -= h
                fd[j] = (_loss(O, rob, *ap, *ups) - _loss(O, rob, *am, *ups)) / (2 * h)
            assert np.abs(g[:, b] - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("mk", [R.r7, R.mixed_joint_tree, R.r23])
def test_fd_gradient_matches_dual_gradient(oracle_lib, mk):
    """The central-difference gradient of full forward evaluations (the CPU
    fwd + bwd the benchmark times) equals the dual-number gradient, with
    d_min as the minimum over every pair, at configurations whose worst pair
    stays the minimum within the step."""
    O = oracle_lib
    rob = mk()
    B = 4
    q, qd, qdd = states(rob, B, 81)
    gp, gs, gm, gt = I.upstream_grads(rob, B, 82)
    dual = O.gradient(rob, q, qd, qdd, gp, gs, gm, gt, nthreads=1)
    fd = O.gradient_fd(rob, q, qd, qdd, gp, gs, gm, gt, h=1e-6, nthreads=2)
    for g, f in zip(dual, fd):
        scale = np.maximum(np.abs(g).max(axis=0), 1.0)
        assert (np.abs(g - f).max(axis=0) <= 1e-7 * scale).all()
    with pytest.raises(ValueError):
        O.gradient_fd(rob, q, qd, qdd, gp, gs, gm, gt, h=0.0)


# ---------------------------------------------------------------------------
# B-spline (Sec. 4)
# ---------------------------------------------------------------------------

def test_bspline_reproduces_polynomials(oracle_lib):
    """Uniform cubic B-splines reproduce constants and lines exactly, and for
    control points u_i = i^2 give (i+1+alpha)^2 + 1/3; derivatives scale by
    1/dt per order."""
    O = oracle_lib
    K, T, dt = 16, 64, 0.25
    idx = np.arange(K, dtype=float)
    U = np.stack([np.full(K, 0.7), 0.3 + 0.5 * idx, idx ** 2])[None]
    q, qd, qdd = O.bspline(U, T, dt)
    nseg = K - 3
    t = np.arange(T) * nseg / (T - 1)
    k = np.minimum(np.floor(t), nseg - 1)
    alpha = t - k
    x = k + 1 + alpha
    assert np.allclose(q[0], 0.7, atol=1e-14) and np.allclose(qd[0], 0, atol=1e-13)
    assert np.allclose(q[1], 0.3 + 0.5 * x, atol=1e-13)
    assert np.allclose(qd[1], 0.5 / dt, atol=1e-12) and np.allclose(qdd[1], 0, atol=1e-11)
    assert np.allclose(q[2], x ** 2 + 1.0 / 3.0, atol=1e-12)
    assert np.allclose(qd[2], 2 * x / dt, atol=1e-11)
    assert np.allclose(qdd[2], 2 / dt ** 2, atol=1e-10)


def _golden_bspline():
    """The paper's printed B-spline tables (tests/golden/bspline_cubic.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "bspline_cubic.txt")
    blocks, cur = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line[0].isalpha():  # a table name
                cur = blocks.setdefault(line, [])
                continue
            cur.append([float(x) for x in line.split()])
    return np.array(blocks["C6"]) / 6.0, np.array(blocks["GHOST"])


def test_bspline_matches_the_printed_coefficients(oracle_lib):
    """Eq. bspline-cubic with the C matrix the paper prints: probing the
    oracle with unit control vectors on one segment recovers, for every
    sample, the 3 x 4 map from the window's control points to (q, qd, qdd),
    and it equals the first three rows of T P(alpha) C."""
    O = oracle_lib
    C, _ = _golden_bspline()
    assert C.shape == (4, 4)
    K, T, dt = 4, 9, 0.37
    cols = []
    for l in range(K):
        U = np.zeros((1, 1, K))
        U[0, 0, l] = 1.0
        q, qd, qdd = O.bspline(U, T, dt)
        cols.append(np.stack([q[0], qd[0], qdd[0]]))  # [3][T]
    M = np.stack(cols, axis=-1)  # [3][T][4]
    for s in range(T):
        a = s / (T - 1)  # one segment: t = alpha
        P = np.array([[a ** 3, a ** 2, a, 1.0],
                      [3 * a ** 2, 2 * a, 1.0, 0.0],
                      [6 * a, 2.0, 0.0, 0.0]])
        Tm = np.diag([1.0, 1.0 / dt, 1.0 / dt ** 2])
        assert np.allclose(M[:, s, :], Tm @ P @ C, atol=1e-13)


def test_bspline_ghost_knots_match_the_printed_coefficients(oracle_lib):
    """Eqs. fixed_3, fixed_2, fixed_1 as printed: probing ghost_knots with a
    unit theta_0, thetadot_0 and thetaddot_0 recovers the coefficients of
    each ghost control point."""
    O = oracle_lib
    _, G = _golden_bspline()
    dt = 0.29
    for i, cv, num, den in G:
        slot = 3 - int(i)  # u_-3, u_-2, u_-1 in order
        for comp, want in ((0, 1.0), (1, cv * dt), (2, num / den * dt * dt)):
            st = np.zeros((1, 1, 3))
            st[0, 0, comp] = 1.0
            assert abs(O.ghost_knots(st, dt)[0, 0, slot] - want) < 1e-15


def test_bspline_vjp_is_the_adjoint(oracle_lib):
    """The B-spline map U -> (q, qd, qdd) is linear, so its VJP must satisfy
    <bspline(U), g> = <U, vjp(g)> for every U and g (Eq. backward_grad is the
    transpose of Eq. bspline-cubic)."""
    O = oracle_lib
    rng = np.random.default_rng(31)
    n_traj, d, K, T, dt = 3, 4, 9, 23, 0.3
    U = rng.normal(size=(n_traj, d, K))
    g = [rng.normal(size=(d, n_traj * T)) for _ in range(3)]
    q, qd, qdd = O.bspline(U, T, dt)
    lhs = sum(float((a * b).sum()) for a, b in zip((q, qd, qdd), g))
    Ub = O.bspline_vjp(*g, n_traj, K, T, dt)
    assert abs(lhs - float((U * Ub).sum())) <= 1e-11 * max(1.0, abs(lhs))
    # each upstream array alone, the others absent
    for i in range(3):
        gi = [g[k] if k == i else None for k in range(3)]
        Ui = O.bspline_vjp(*gi, n_traj, K, T, dt)
        lhs_i = float(((q, qd, qdd)[i] * g[i]).sum())
        assert abs(lhs_i - float((U * Ui).sum())) <= 1e-11 * max(1.0, abs(lhs_i))


def test_bspline_vjp_local_support_is_the_textbook_basis(oracle_lib):
    """A unit gradient on one sample's position reaches only the four control
    points of its window, with the uniform cubic B-spline basis values
    (1-a)^3/6, (3a^3-6a^2+4)/6, (-3a^3+3a^2+3a+1)/6, a^3/6 (partition of
    unity); on its velocity, their derivatives / dt."""
    O = oracle_lib
    K, T, dt = 10, 19, 0.2
    nseg = K - 3
    for s in (0, 5, 11, T - 1):
        t = s * nseg / (T - 1)
        k = min(int(np.floor(t)), nseg - 1)
        a = t - k
        g = np.zeros((1, T))
        g[0, s] = 1.0
        Ub = O.bspline_vjp(g, None, None, 1, K, T, dt)[0, 0]
        basis = np.array([(1 - a) ** 3, 3 * a ** 3 - 6 * a ** 2 + 4,
                          -3 * a ** 3 + 3 * a ** 2 + 3 * a + 1, a ** 3]) / 6
        ref = np.zeros(K)
        ref[k:k + 4] = basis
        assert np.allclose(Ub, ref, atol=1e-14)
        assert abs(basis.sum() - 1.0) < 1e-14
        Ubd = O.bspline_vjp(None, g, None, 1, K, T, dt)[0, 0]
        dbasis = np.array([-3 * (1 - a) ** 2, 9 * a ** 2 - 12 * a, -9 * a ** 2 + 6 * a + 3,
                           3 * a ** 2]) / 6 / dt
        refd = np.zeros(K)
        refd[k:k + 4] = dbasis
        assert np.allclose(Ubd, refd, atol=1e-13)


def test_trajopt_chain_with_summed_hinge_matches_finite_differences(oracle_lib):
    """The chain with the summed collision hinge (every masked pair within
    the activation distance) and the motion terms: its gradient, with the
    hinge's sphere-centre gradient fed to the whole-body VJP, equals central
    differences of the total cost."""
    O = oracle_lib
    rob = R.r7()
    rng = np.random.default_rng(19)
    n_traj, K, T, dt = 2, 6, 9, 0.25
    U = rng.uniform(-1.5, 1.5, size=(n_traj, rob.dof, K))
    lo, hi = -8.0 * np.ones(rob.dof), 8.0 * np.ones(rob.dof)
    kw = dict(smooth=0.01, length=0.1, energy=0.05, eta=0.05)
    Ub, cost, _ = O.trajopt_gradient(rob, U, T, dt, lo, hi, 2.0, **kw)
    q, _, _ = O.bspline(U, T, dt)
    hc, _ = O.pair_hinge(rob, q, 0.05, 2.0)
    assert (hc > 0).mean() > 0.5  # the hinge is active on most samples
    h = 1e-6
    for flat in rng.choice(U.size, size=10, replace=False):
        idx = np.unravel_index(flat, U.shape)
        Up, Um = U.copy(), U.copy()
        Up[idx] += h
        Um[idx] -= h
        fd = (O.trajopt_value(rob, Up, T, dt, lo, hi, 2.0, **kw)[0] -
              O.trajopt_value(rob, Um, T, dt, lo, hi, 2.0, **kw)[0]) / (2 * h)
        assert abs(fd - Ub[idx]) <= 1e-6 * max(1.0, abs(Ub[idx])), (idx, fd, Ub[idx])


def test_bspline_ghost_knots_continue_the_start_state(oracle_lib):
    """With a non-static start (Sec. 4.2) the first sampled window is
    [u_-3, u_-2, u_-1, u_0]; its state at alpha = 0 depends on the ghost
    knots only and is the start state carried one knot interval forward with
    zero jerk: q = th0 + v dt + a dt^2 / 2, qd = v + a dt, qdd = a, whatever
    the optimised control points.  Three equations in the three ghost knots,
    so a wrong coefficient in any of them shows here."""
    O = oracle_lib
    rng = np.random.default_rng(41)
    n_traj, d, K, T, dt = 3, 5, 8, 12, 0.3
    start = rng.normal(size=(n_traj, d, 3))
    th, v, a = start[..., 0], start[..., 1], start[..., 2]
    for seed in (1, 2):
        U = np.random.default_rng(seed).normal(size=(n_traj, d, K))
        for end in (False, True):
            q, qd, qdd = O.bspline_bc(U, T, dt, start=start, end_static=end)
            first = np.arange(n_traj) * T  # sample 0 of each trajectory
            assert np.allclose(q[:, first].T, th + v * dt + a * dt * dt / 2, atol=1e-13)
            assert np.allclose(qd[:, first].T, v + a * dt, atol=1e-12)
            assert np.allclose(qdd[:, first].T, a, atol=1e-11)


def test_bspline_static_goal_stops_at_the_last_control_point(oracle_lib):
    """Repeating the final control point until it appears four times (Sec.
    4.2) makes the last segment constant: the final sample is at u_K-1 with
    zero velocity and acceleration (Eq. stop-constraint), and so is every
    sample of that segment."""
    O = oracle_lib
    rng = np.random.default_rng(42)
    n_traj, d, K, T, dt = 2, 4, 9, 25, 0.2
    U = rng.normal(size=(n_traj, d, K))
    for start in (None, rng.normal(size=(n_traj, d, 3))):
        q, qd, qdd = O.bspline_bc(U, T, dt, start=start, end_static=True)
        nseg = K + 3 + (3 if start is not None else 0) - 3
        t = np.arange(T) * nseg / (T - 1)
        last = t >= nseg - 1  # samples inside the final segment
        assert last.sum() >= 2
        for tr in range(n_traj):
            sl = np.arange(tr * T, (tr + 1) * T)[last]
            assert np.allclose(q[:, sl], U[tr, :, -1:], atol=1e-13)
            assert np.allclose(qd[:, sl], 0.0, atol=1e-12)
            assert np.allclose(qdd[:, sl], 0.0, atol=1e-11)


def test_bspline_boundary_vjp_is_the_adjoint(oracle_lib):
    """q, qd, qdd are linear in (U, start state) together, so the VJP with the
    repeated final knots folded onto u_K-1 and the start-state gradient
    through the ghost knots must satisfy <g, states> = <gU, U> + <gs, start>;
    and a unit gradient on the first sample's position reaches the start
    state only, as d q / d (th0, v, a) = (1, dt, dt^2 / 2)."""
    O = oracle_lib
    rng = np.random.default_rng(43)
    n_traj, d, K, T, dt = 3, 4, 7, 17, 0.25
    U = rng.normal(size=(n_traj, d, K))
    start = rng.normal(size=(n_traj, d, 3))
    g = [rng.normal(size=(d, n_traj * T)) for _ in range(3)]
    for has_start in (False, True):
        for end in (False, True):
            st = start if has_start else None
            states = O.bspline_bc(U, T, dt, start=st, end_static=end)
            lhs = sum(float((a * b).sum()) for a, b in zip(states, g))
            gU, gs = O.bspline_bc_vjp(*g, n_traj, K, T, dt, has_start=has_start,
                                      end_static=end)
            rhs = float((U * gU).sum()) + (float((start * gs).sum()) if has_start else 0.0)
            assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs)), (has_start, end)
            assert (gs is None) == (not has_start)
    g0 = np.zeros((d, n_traj * T))
    g0[2, T] = 1.0  # joint 2, trajectory 1, sample 0
    gU, gs = O.bspline_bc_vjp(g0, None, None, n_traj, K, T, dt, has_start=True)
    assert np.allclose(gU, 0.0, atol=1e-15)
    ref = np.zeros((n_traj, d, 3))
    ref[1, 2] = [1.0, dt, dt * dt / 2]
    assert np.allclose(gs, ref, atol=1e-14)


def test_trajopt_cost_closed_form(oracle_lib):
    """Hinges on hand-made torques and distances: only the parts beyond the
    limits count, gradients are +-1 there, and the collision hinge is
    -w dmin for penetration only."""
    O = oracle_lib
    tau = np.array([[35.0, 10.0, -31.0], [-40.0, 29.9, 0.0]])  # [d=2][B=3]
    dmin = np.array([0.2, -0.05, 0.0])
    lo, hi = np.array([-30.0, -30.0]), np.array([30.0, 30.0])
    cost, g_tau, g_dmin = O.trajopt_cost(tau, dmin, lo, hi, 2.0)
    assert np.allclose(cost, [5.0 + 10.0, 0.0 + 2.0 * 0.05, 1.0 + 0.0], atol=1e-12)
    assert np.array_equal(g_tau, [[1.0, 0.0, -1.0], [-1.0, 0.0, 0.0]])
    assert np.array_equal(g_dmin, [0.0, -2.0, 0.0])


def test_trajopt_chain_gradient_matches_finite_differences(oracle_lib):
    """dL/dU through cost -> whole-body VJP -> B-spline VJP equals central
    differences of the total cost, at control points where no hinge and no
    worst pair switches within the step (torque limits at the median |tau|,
    sphere radii scaled so that some samples penetrate and some do not)."""
    import dataclasses
    O = oracle_lib
    base = R.r7()
    rob = dataclasses.replace(base, sph_r=base.sph_r * 0.7)
    rng = np.random.default_rng(5)
    n_traj, K, T, dt = 2, 6, 9, 0.25
    U = rng.uniform(-1.5, 1.5, size=(n_traj, rob.dof, K))
    _, ev = O.trajopt_value(rob, U, T, dt, -np.ones(rob.dof), np.ones(rob.dof), 1.0)
    lim = float(np.median(np.abs(ev["tau"])))
    lo, hi, w = -lim * np.ones(rob.dof), lim * np.ones(rob.dof), 1.5
    assert (ev["dmin"] < 0).any() and (ev["dmin"] > 0).any()
    Ub, cost, ev = O.trajopt_gradient(rob, U, T, dt, lo, hi, w)
    assert ((np.abs(ev["tau"]) > lim).mean()) > 0.2
    h = 1e-6
    checked = 0
    for flat in rng.choice(U.size, size=16, replace=False):
        idx = np.unravel_index(flat, U.shape)
        Up, Um = U.copy(), U.copy()
        Up[idx] += h
        Um[idx] -= h
        vp, evp = O.trajopt_value(rob, Up, T, dt, lo, hi, w)
        vm, evm = O.trajopt_value(rob, Um, T, dt, lo, hi, w)
        same = all(np.array_equal(a["tau"] > hi[:, None], ev["tau"] > hi[:, None]) and
                   np.array_equal(a["tau"] < lo[:, None], ev["tau"] < lo[:, None]) and
                   np.array_equal(a["dmin"] < 0, ev["dmin"] < 0) and
                   np.array_equal(a["worst"], ev["worst"]) for a in (evp, evm))
        if not same:
            continue
        fd = (vp - vm) / (2 * h)
        assert abs(fd - Ub[idx]) <= 1e-6 * max(1.0, abs(Ub[idx])), (idx, fd, Ub[idx])
        checked += 1
    assert checked >= 8


def test_pair_hinge_hand_built(oracle_lib):
    """Three slider spheres (centres (q_k, 0, 0)): every pair closer than the
    activation distance adds w (eta - d); the gradient pushes each sphere of
    an active pair away from its partner with weight w; since each slider
    moves its sphere along x, the joint gradient is the x component."""
    O = oracle_lib
    rob = _slider_robot([0.25, 0.125, 0.5])
    q = np.array([[0.0], [0.375], [0.5]])
    eta, w = 0.1, 2.0
    # d01 = 0.375 - 0.375 = 0, d02 = 0.5 - 0.75 = -0.25, d12 = 0.125 - 0.625 = -0.5
    cost, g = O.pair_hinge(rob, q, eta, w)
    assert cost[0] == pytest.approx(w * (0.1 + 0.35 + 0.6), abs=1e-15)
    # sphere 0 is left of both partners, sphere 2 right of both, sphere 1 between
    assert np.allclose(g[0, :, 0], [w * 2, w * (-1 + 1), -w * 2], atol=1e-15)
    assert np.allclose(g[0, :, 1:], 0.0)
    gq, _, _ = O.gradient(rob, q, np.zeros_like(q), np.zeros_like(q), g_sph=g)
    assert np.allclose(gq[:, 0], g[0, :, 0], atol=1e-14)
    # move sphere 2 far away: only pair (0, 1) stays active; at d = eta exactly
    # nothing is added
    cost, g = O.pair_hinge(rob, np.array([[0.0], [0.375], [5.0]]), eta, w)
    assert cost[0] == pytest.approx(w * 0.1) and np.allclose(g[0, 2], 0.0)
    cost, g = O.pair_hinge(rob, np.array([[0.0], [0.5], [5.0]]), 0.125, w)  # d01 = 0.125 exactly
    assert cost[0] == 0.0 and np.allclose(g, 0.0)


def test_pair_hinge_gradient_matches_finite_differences(oracle_lib):
    """d(cost)/dq through the sphere gradient and the whole-body VJP equals
    central differences of the summed hinge on the 7-DoF chain, at
    configurations where no pair crosses the activation distance within the
    step."""
    O = oracle_lib
    rob = R.r7()
    rng = np.random.default_rng(12)
    q = rng.uniform(-np.pi, np.pi, size=(rob.dof, 6))
    eta, w, h = 0.05, 1.7, 1e-6
    cost, g = O.pair_hinge(rob, q, eta, w)
    assert (cost > 0).all()
    gq, _, _ = O.gradient(rob, q, np.zeros_like(q), np.zeros_like(q), g_sph=g)
    fd = np.zeros_like(q)
    for j in range(rob.dof):
        qp, qm = q.copy(), q.copy()
        qp[j] += h
        qm[j] -= h
        fd[j] = (O.pair_hinge(rob, qp, eta, w)[0] - O.pair_hinge(rob, qm, eta, w)[0]) / (2 * h)
    assert np.allclose(gq, fd, rtol=1e-6, atol=1e-6)


def test_jacobian_and_com_planar_closed_form(oracle_lib):
    """2-link planar arm (axes z, link 2 at (l1, 0, 0), unit masses with CoMs
    at the link midpoints (l1/2, 0, 0) and (l2/2, 0, 0)): link 2's origin
    (l1 c1, l1 s1) moves with (-l1 s1, l1 c1) under q1 and not under q2; both
    columns turn about z; the CoM is the mean of the two link CoMs."""
    O = oracle_lib
    l1, l2 = 0.5, 0.25
    rob = R.planar_2link(l1, l2)
    q1, q2 = 0.3, 0.5
    J, com, Jc = O.kinematics(rob, np.array([[q1], [q2]]), [0, 1])
    c1, s1, c12, s12 = np.cos(q1), np.sin(q1), np.cos(q1 + q2), np.sin(q1 + q2)
    ref1 = np.array([[-l1 * s1, 0], [l1 * c1, 0], [0, 0], [0, 0], [0, 0], [1, 1]])
    assert np.allclose(J[0, 1], ref1, atol=1e-14)
    assert np.allclose(J[0, 0], [[0, 0]] * 5 + [[1, 0]], atol=1e-14)  # link 1 at the origin
    m1 = np.array([l1 / 2 * c1, l1 / 2 * s1, 0.0])
    m2 = np.array([l1 * c1 + l2 / 2 * c12, l1 * s1 + l2 / 2 * s12, 0.0])
    assert np.allclose(com[0], (m1 + m2) / 2, atol=1e-15)
    dm1 = np.array([[-l1 / 2 * s1, 0], [l1 / 2 * c1, 0], [0, 0]])
    dm2 = np.array([[-l1 * s1 - l2 / 2 * s12, -l2 / 2 * s12],
                    [l1 * c1 + l2 / 2 * c12, l2 / 2 * c12], [0, 0]])
    assert np.allclose(Jc[0], (dm1 + dm2) / 2, atol=1e-15)


def test_jacobian_and_com_match_finite_differences(oracle_lib):
    """On the humanoid with hand payloads: linear rows = central differences
    of the link origins, angular rows = vee(dR R^T) by central differences of
    the rotations; the CoM equals the mass-weighted sum over link CoMs and
    point masses from the poses, and its Jacobian its central differences."""
    O = oracle_lib
    rob = I.hand_payload(R.r48())
    rng = np.random.default_rng(21)
    q = rng.uniform(-np.pi, np.pi, size=(rob.dof, 2))
    targets = [0, 11, 27, rob.n - 1]
    J, com, Jc = O.kinematics(rob, q, targets)

    def poses(qq):
        return O.evaluate(rob, qq, want=("pose",))["pose"]

    def com_from(P):
        m = np.concatenate([rob.mass, rob.pm_mass])
        links = np.concatenate([np.arange(rob.n), rob.pm_link])
        loc = np.concatenate([rob.com, rob.pm_pos])
        R3 = P[:, links, :9].reshape(-1, len(links), 3, 3)
        x = np.einsum("blij,lj->bli", R3, loc) + P[:, links, 9:]
        return (m[None, :, None] * x).sum(axis=1) / m.sum()
    P0 = poses(q)
    assert np.allclose(com, com_from(P0), atol=1e-13)
    h = 1e-6
    for j in range(0, rob.dof, 7):
        qp, qm = q.copy(), q.copy()
        qp[j] += h
        qm[j] -= h
        Pp, Pm = poses(qp), poses(qm)
        for t, e in enumerate(targets):
            lin = (Pp[:, e, 9:] - Pm[:, e, 9:]) / (2 * h)
            assert np.allclose(J[:, t, :3, j], lin, atol=1e-7)
            dR = (Pp[:, e, :9] - Pm[:, e, :9]).reshape(-1, 3, 3) / (2 * h)
            Wm = dR @ P0[:, e, :9].reshape(-1, 3, 3).transpose(0, 2, 1)
            ang = np.stack([Wm[:, 2, 1], Wm[:, 0, 2], Wm[:, 1, 0]], axis=1)
            assert np.allclose(J[:, t, 3:, j], ang, atol=1e-7)
        assert np.allclose(Jc[:, :, j], (com_from(Pp) - com_from(Pm)) / (2 * h), atol=1e-7)


def _support_forces(rob, P):
    """Per link, the wrench (link coordinates, moment then force, about the
    link origin) that holds its mass and payload point masses against
    gravity: force m R^T (-g) at each mass point."""
    B = P.shape[0]
    f = np.zeros((B, rob.n, 6))
    pts = [(k, rob.mass[k], rob.com[k]) for k in range(rob.n)]
    pts += [(int(l), m, x) for l, m, x in zip(rob.pm_link, rob.pm_mass, rob.pm_pos)]
    g = np.asarray(rob.gravity, float)
    for k, m, x in pts:
        Rk = P[:, k, :9].reshape(B, 3, 3)
        F = m * np.einsum("bji,j->bi", Rk, -g)
        f[:, k, 3:] += F
        f[:, k, :3] += np.cross(np.broadcast_to(x, F.shape), F)
    return f


def test_external_support_forces_cancel_gravity(oracle_lib):
    """External forces that hold every link up against gravity leave zero
    joint torque at rest, in any configuration (sign, frame and moment-first
    ordering of f_ext)."""
    O = oracle_lib
    rob = I.hand_payload(R.r48())
    rng = np.random.default_rng(8)
    q = rng.uniform(-np.pi, np.pi, size=(rob.dof, 3))
    P = O.evaluate(rob, q, want=("pose",))["pose"]
    z = np.zeros_like(q)
    tau0 = O.evaluate(rob, q, z, z, want=("tau",))["tau"]
    assert np.abs(tau0).max() > 10.0
    tau = O.evaluate(rob, q, z, z, fext=_support_forces(rob, P), want=("tau",))["tau"]
    assert np.abs(tau).max() < 1e-10


def test_fext_gradient_is_minus_the_link_frame_jacobian(oracle_lib):
    """d tau_j / d f_ext,k = -(link k's origin Jacobian column j in link k's
    coordinates, angular then linear): the transpose of the kinematics that
    maps joint rates to link k's twist."""
    O = oracle_lib
    rob = R.r23()
    rng = np.random.default_rng(4)
    B = 2
    q, qd, qdd = (rng.uniform(-2, 2, size=(rob.dof, B)) for _ in range(3))
    fext = rng.normal(size=(B, rob.n, 6))
    J, _, _ = O.kinematics(rob, q, list(range(rob.n)))
    P = O.evaluate(rob, q, want=("pose",))["pose"]
    for j in (0, 5, rob.dof - 1):
        gt = np.zeros((rob.dof, B))
        gt[j] = 1.0
        g = O.fext_gradient(rob, q, qd, qdd, fext, gt)
        for k in range(rob.n):
            Rk = P[:, k, :9].reshape(B, 3, 3)
            ang = np.einsum("bji,bj->bi", Rk, J[:, k, 3:, j])
            lin = np.einsum("bji,bj->bi", Rk, J[:, k, :3, j])
            assert np.allclose(g[:, k], -np.concatenate([ang, lin], axis=1), atol=1e-9)


def test_motion_cost_terms_closed_form(oracle_lib):
    """smooth |qdd|^2 + length |qd|^2 + energy ||(qd . tau) dt||^2 on hand
    numbers, with their tau / qd / qdd gradients."""
    O = oracle_lib
    tau = np.array([[2.0], [-3.0]])
    qd = np.array([[0.5], [4.0]])
    qdd = np.array([[1.0], [-2.0]])
    lo, hi = np.array([-10.0, -10.0]), np.array([10.0, 10.0])
    cost, g_tau, g_dmin, g_qd, g_qdd = O.trajopt_cost(tau, np.array([1.0]), lo, hi, 1.0, qd, qdd,
                                                      smooth=0.5, length=0.25, energy=2.0,
                                                      dt=0.1)
    # smooth 0.5 (1 + 4) = 2.5; length 0.25 (0.25 + 16) = 4.0625;
    # energy 2 * 0.01 * ((0.5 * 2)^2 + (4 * -3)^2) = 0.02 * 145 = 2.9
    assert cost[0] == pytest.approx(2.5 + 4.0625 + 2.9, abs=1e-12)
    e = 2.0 * 0.01
    assert np.allclose(g_tau[:, 0], [2 * e * 0.25 * 2.0, 2 * e * 16.0 * -3.0], atol=1e-12)
    assert np.allclose(g_qd[:, 0], [2 * 0.25 * 0.5 + 2 * e * 0.5 * 4.0,
                                    2 * 0.25 * 4.0 + 2 * e * 4.0 * 9.0], atol=1e-12)
    assert np.allclose(g_qdd[:, 0], [1.0, -2.0], atol=1e-12)
    assert g_dmin[0] == 0.0


def test_trajopt_chain_with_motion_terms_matches_finite_differences(oracle_lib):
    """The chain gradient with smooth, length and energy terms (their direct
    qd / qdd gradients added before the B-spline VJP) equals central
    differences of the total cost."""
    O = oracle_lib
    rob = R.r7()
    rng = np.random.default_rng(9)
    n_traj, K, T, dt = 2, 6, 9, 0.25
    U = rng.uniform(-1.0, 1.0, size=(n_traj, rob.dof, K))
    lo, hi = -1e3 * np.ones(rob.dof), 1e3 * np.ones(rob.dof)  # hinges inactive
    kw = dict(smooth=0.01, length=0.1, energy=0.05)
    Ub, _, _ = O.trajopt_gradient(rob, U, T, dt, lo, hi, 0.0, **kw)
    h = 1e-6
    for flat in rng.choice(U.size, size=10, replace=False):
        idx = np.unravel_index(flat, U.shape)
        Up, Um = U.copy(), U.copy()
        Up[idx] += h
        Um[idx] -= h
        fd = (O.trajopt_value(rob, Up, T, dt, lo, hi, 0.0, **kw)[0] -
              O.trajopt_value(rob, Um, T, dt, lo, hi, 0.0, **kw)[0]) / (2 * h)
        assert abs(fd - Ub[idx]) <= 1e-6 * max(1.0, abs(Ub[idx])), (idx, fd, Ub[idx])
