"""ctypes wrapper around the FP64 CPU oracle (wb_oracle.cpp).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It does not import the CUDA library
and the CUDA library does not import it.

Arrays cross this wrapper in the library's layouts (q, qd, qdd, tau as [d][B];
poses [B][n][12]; spheres [B][S][3]) and are converted to the oracle's
config-major float64 layout here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wb_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "libwb_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ -O3 (plain double; OpenMP across
    configurations)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _OUT)
    return _OUT


class _Robot(C.Structure):
    _fields_ = [("n", C.c_int), ("d", C.c_int), ("S", C.c_int), ("P", C.c_int),
                ("n_pm", C.c_int),
                ("parent", C.c_void_p), ("jtype", C.c_void_p), ("axis", C.c_void_p),
                ("T_fixed", C.c_void_p), ("jidx", C.c_void_p), ("mimic_mult", C.c_void_p),
                ("mimic_off", C.c_void_p), ("gravity", C.c_void_p), ("sph_link", C.c_void_p),
                ("sph_c", C.c_void_p), ("sph_r", C.c_void_p), ("pairs", C.c_void_p),
                ("mass", C.c_void_p), ("com", C.c_void_p), ("Icom", C.c_void_p),
                ("pm_link", C.c_void_p), ("pm_mass", C.c_void_p), ("pm_pos", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        p = C.c_void_p
        _lib.or_eval.argtypes = [C.POINTER(_Robot), C.c_int, p, p, p, p, p, p, p, p, p, p, C.c_int]
        _lib.or_grad.argtypes = [C.POINTER(_Robot), C.c_int, p, p, p, p, p, p, p, p, p, p, p,
                                 C.c_int]
        _lib.or_grad_fd.argtypes = [C.POINTER(_Robot), C.c_int, p, p, p, p, p, p, p, p,
                                    C.c_double, p, p, p, C.c_int]
        _lib.or_bspline.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, p, p, p, p]
        _lib.or_bspline_vjp.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, p, p, p,
                                        p]
        _lib.or_kinematics.argtypes = [C.POINTER(_Robot), C.c_int, p, C.c_int, p, p, p, p,
                                       C.c_int]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleRobot:
    """Holds contiguous float64/int32 copies of a synthetic Robot."""

    def __init__(self, robot):
        self.robot = robot
        self._keep = {}

        def keep(name, a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep[name] = a
            return a.ctypes.data

        r = robot
        s = _Robot()
        s.n, s.d, s.S, s.P, s.n_pm = r.n, r.dof, r.S, r.P, len(r.pm_link)
        s.parent = keep("parent", r.parent, np.int32)
        s.jtype = keep("jtype", r.jtype, np.int32)
        s.axis = keep("axis", r.axis, np.float64)
        s.T_fixed = keep("T", r.T_fixed, np.float64)
        s.jidx = keep("jidx", r.jidx, np.int32)
        s.mimic_mult = keep("mm", r.mimic_mult, np.float64)
        s.mimic_off = keep("mo", r.mimic_off, np.float64)
        s.gravity = keep("g", r.gravity, np.float64)
        s.sph_link = keep("sl", r.sph_link, np.int32)
        s.sph_c = keep("sc", r.sph_c, np.float64)
        s.sph_r = keep("sr", r.sph_r, np.float64)
        s.pairs = keep("pairs", r.pairs.reshape(-1, 2) if r.P else np.zeros((1, 2)), np.int32)
        s.mass = keep("mass", r.mass, np.float64)
        s.com = keep("com", r.com, np.float64)
        s.Icom = keep("Icom", r.Icom, np.float64)
        s.pm_link = keep("pml", r.pm_link if len(r.pm_link) else np.zeros(1), np.int32)
        s.pm_mass = keep("pmm", r.pm_mass if len(r.pm_mass) else np.zeros(1), np.float64)
        s.pm_pos = keep("pmp", r.pm_pos if len(r.pm_pos) else np.zeros((1, 3)), np.float64)
        self.s = s


def _cm(x, d):
    """[d][B] (library layout) -> contiguous float64 [B][d]."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(d, -1).T)


def evaluate(robot, q, qd=None, qdd=None, fext=None, want=("pose", "sph", "dmin", "tau"),
             nthreads: int = 0):
    """Forward evaluation.  q, qd, qdd in [d][B].  Returns a dict with
    pose [B][n][12], sph [B][S][3], dmin [B], worst [B], collide [B][P] uint8,
    tau [d][B] (each only if in `want`)."""
    orob = robot if isinstance(robot, OracleRobot) else OracleRobot(robot)
    r = orob.robot
    d = r.dof
    q = _cm(q, d)
    B = q.shape[0]
    need_tau = "tau" in want
    qd = _cm(qd, d) if qd is not None else np.zeros_like(q)
    qdd = _cm(qdd, d) if qdd is not None else np.zeros_like(q)
    out = {}
    pose = np.zeros((B, r.n, 12)) if "pose" in want else None
    sph = np.zeros((B, r.S, 3)) if "sph" in want else None
    need_pair = "dmin" in want or "worst" in want or "collide" in want
    dmin = np.zeros(B) if need_pair else None
    worst = np.zeros(B, np.int32) if need_pair else None
    collide = np.zeros((B, max(r.P, 1)), np.uint8) if "collide" in want else None
    tau = np.zeros((B, d)) if need_tau else None
    fe = None if fext is None else np.ascontiguousarray(fext, dtype=np.float64)
    lib().or_eval(C.byref(orob.s), B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(fe), _ptr(pose),
                  _ptr(sph), _ptr(dmin), _ptr(worst), _ptr(collide), _ptr(tau), nthreads)
    if pose is not None:
        out["pose"] = pose
    if sph is not None:
        out["sph"] = sph
    if need_pair:
        out["dmin"] = dmin
        out["worst"] = worst
    if collide is not None:
        out["collide"] = collide[:, :r.P]
    if tau is not None:
        out["tau"] = np.ascontiguousarray(tau.T)
    return out


def gradient(robot, q, qd, qdd, g_pose=None, g_sph=None, g_dmin=None, g_tau=None, fext=None,
             nthreads: int = 0):
    """Exact (dual-number) gradient of <g_pose,pose> + <g_sph,sph> +
    g_dmin*d_min + <g_tau,tau> w.r.t. q, qd, qdd.  Inputs in library layouts;
    returns (gq, gqd, gqdd) each [d][B]."""
    orob = robot if isinstance(robot, OracleRobot) else OracleRobot(robot)
    r = orob.robot
    d = r.dof
    q = _cm(q, d)
    B = q.shape[0]
    qd = _cm(qd, d)
    qdd = _cm(qdd, d)
    gp = None if g_pose is None else np.ascontiguousarray(g_pose, dtype=np.float64)
    gs = None if g_sph is None else np.ascontiguousarray(g_sph, dtype=np.float64)
    gm = None if g_dmin is None else np.ascontiguousarray(g_dmin, dtype=np.float64)
    gt = None if g_tau is None else _cm(g_tau, d)
    fe = None if fext is None else np.ascontiguousarray(fext, dtype=np.float64)
    gq = np.zeros((B, d))
    gqd = np.zeros((B, d))
    gqdd = np.zeros((B, d))
    lib().or_grad(C.byref(orob.s), B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(fe), _ptr(gp),
                  _ptr(gs), _ptr(gm), _ptr(gt), _ptr(gq), _ptr(gqd), _ptr(gqdd), nthreads)
    return (np.ascontiguousarray(gq.T), np.ascontiguousarray(gqd.T),
            np.ascontiguousarray(gqdd.T))


def gradient_fd(robot, q, qd, qdd, g_pose=None, g_sph=None, g_dmin=None, g_tau=None,
                fext=None, h: float = 1e-6, nthreads: int = 0):
    """The gradient of `gradient`'s loss by central differences of full
    forward evaluations (or_grad_fd: 2*3d forward evaluations per
    configuration, d_min as the minimum over every pair; with the forward
    evaluation at the point, 2*3d + 1).  Valid away from kinks of the
    minimum.  Returns (gq, gqd, gqdd) each [d][B]."""
    orob = robot if isinstance(robot, OracleRobot) else OracleRobot(robot)
    r = orob.robot
    d = r.dof
    q = _cm(q, d)
    B = q.shape[0]
    qd = _cm(qd, d)
    qdd = _cm(qdd, d)
    gp = None if g_pose is None else np.ascontiguousarray(g_pose, dtype=np.float64)
    gs = None if g_sph is None else np.ascontiguousarray(g_sph, dtype=np.float64)
    gm = None if g_dmin is None else np.ascontiguousarray(g_dmin, dtype=np.float64)
    gt = None if g_tau is None else _cm(g_tau, d)
    fe = None if fext is None else np.ascontiguousarray(fext, dtype=np.float64)
    gq = np.zeros((B, d))
    gqd = np.zeros((B, d))
    gqdd = np.zeros((B, d))
    rc = lib().or_grad_fd(C.byref(orob.s), B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(fe), _ptr(gp),
                          _ptr(gs), _ptr(gm), _ptr(gt), float(h), _ptr(gq), _ptr(gqd),
                          _ptr(gqdd), nthreads)
    if rc != 0:
        raise ValueError("or_grad_fd: h must be positive")
    return (np.ascontiguousarray(gq.T), np.ascontiguousarray(gqd.T),
            np.ascontiguousarray(gqdd.T))


def bspline(U, T: int, dt: float):
    """Uniform cubic B-spline states from control points U [n_traj][d][K].
    Returns q, qd, qdd in [d][n_traj*T]."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    n_traj, d, K = U.shape
    B = n_traj * T
    q = np.zeros((B, d))
    qd = np.zeros((B, d))
    qdd = np.zeros((B, d))
    rc = lib().or_bspline(n_traj, d, K, T, dt, _ptr(U), _ptr(q), _ptr(qd), _ptr(qdd))
    if rc != 0:
        raise ValueError("or_bspline: bad sizes")
    return (np.ascontiguousarray(q.T), np.ascontiguousarray(qd.T), np.ascontiguousarray(qdd.T))


def bspline_vjp(gq, gqd, gqdd, n_traj: int, K: int, T: int, dt: float):
    """Control-point gradient of a scalar with upstream gradients gq, gqd,
    gqdd [d][n_traj*T] on the B-spline states (Eq. backward_grad; each may be
    None).  Returns Ubar [n_traj][d][K]."""
    g = [None if x is None else np.ascontiguousarray(np.asarray(x, np.float64).T)
         for x in (gq, gqd, gqdd)]
    d = next(x.shape[1] for x in g if x is not None)
    Ub = np.zeros((n_traj, d, K))
    rc = lib().or_bspline_vjp(n_traj, d, K, T, dt, _ptr(g[0]), _ptr(g[1]), _ptr(g[2]), _ptr(Ub))
    if rc != 0:
        raise ValueError("or_bspline_vjp: bad sizes")
    return Ub


def ghost_knots(start, dt: float):
    """The three fictitious control points that anchor a spline to a
    non-static initial state (Sec. 4.2, Eqs. fixed_3, fixed_2, fixed_1):
    start [n_traj][d][3] holds theta_0, thetadot_0, thetaddot_0 per joint;
    returns [n_traj][d][3] = u_-3, u_-2, u_-1 with
        u_-3 = theta_0 - thetaddot_0 dt^2 / 6,
        u_-2 = theta_0 + thetadot_0 dt + thetaddot_0 dt^2 / 3,
        u_-1 = theta_0 + 2 thetadot_0 dt + 11 thetaddot_0 dt^2 / 6."""
    st = np.asarray(start, np.float64)
    th, v, a = st[..., 0], st[..., 1], st[..., 2]
    return np.stack([th - a * dt * dt / 6.0,
                     th + v * dt + a * dt * dt / 3.0,
                     th + 2.0 * v * dt + 11.0 * a * dt * dt / 6.0], axis=-1)


def extended_knots(U, start=None, end_static=False, dt: float = 1.0):
    """The knot sequence a boundary-conditioned spline is evaluated on: the
    ghost knots of a non-static start prepended (Sec. 4.2), and for a static
    goal the final control point repeated so that it appears four times
    (Sec. 4.2: the repeated knot makes velocity and acceleration vanish at
    the end, Eq. stop-constraint)."""
    U = np.asarray(U, np.float64)
    parts = []
    if start is not None:
        parts.append(ghost_knots(start, dt))
    parts.append(U)
    if end_static:
        parts.append(np.repeat(U[..., -1:], 3, axis=-1))
    return np.concatenate(parts, axis=-1)


def bspline_bc(U, T: int, dt: float, start=None, end_static=False):
    """B-spline states with boundary conditions: Eq. bspline-cubic evaluated
    on the extended knot sequence (T samples over its segments).  Returns q,
    qd, qdd [d][n_traj*T]."""
    return bspline(extended_knots(U, start, end_static, dt), T, dt)


def bspline_bc_vjp(gq, gqd, gqdd, n_traj: int, K: int, T: int, dt: float, has_start=False,
                   end_static=False):
    """Gradients of a scalar through bspline_bc: the control-point gradient
    [n_traj][d][K] (the VJP on the extended sequence, with the repeated final
    knots folded onto the last control point) and, with a start state, the
    start-state gradient [n_traj][d][3] through the ghost knots (the
    transpose of ghost_knots' linear map)."""
    Kx = K + (3 if has_start else 0) + (3 if end_static else 0)
    gx = bspline_vjp(gq, gqd, gqdd, n_traj, Kx, T, dt)
    o = 3 if has_start else 0
    gU = gx[..., o:o + K].copy()
    if end_static:
        gU[..., -1] += gx[..., o + K:].sum(axis=-1)
    gstart = None
    if has_start:
        g3, g2, g1 = gx[..., 0], gx[..., 1], gx[..., 2]
        gstart = np.stack([g3 + g2 + g1,
                           dt * g2 + 2.0 * dt * g1,
                           dt * dt * (-g3 / 6.0 + g2 / 3.0 + 11.0 * g1 / 6.0)], axis=-1)
    return gU, gstart


def trajopt_cost(tau, dmin, tau_lo, tau_hi, w_coll, qd=None, qdd=None, smooth=0.0,
                 length=0.0, energy=0.0, dt=1.0):
    """Per-configuration cost of the trajectory-optimisation workload and its
    gradients: the motion terms of the problem's loss (Sec. 3,
    Eq. cost_motion_opt), smooth ||qdd||^2,
    length ||qd||^2 and energy ||(qd . tau) dt||^2 with their weights, plus
    the torque-limit hinges per joint and the self-collision hinge on the
    worst pair:
        cost_b = smooth |qdd_b|^2 + length |qd_b|^2
                 + energy dt^2 sum_j (qd_jb tau_jb)^2
                 + sum_j [max(0, tau_jb - hi_j) + max(0, lo_j - tau_jb)]
                 + w max(0, -dmin_b),
        dL/dtau_jb  = 2 energy dt^2 qd_jb^2 tau_jb + [tau_jb > hi_j] - [tau_jb < lo_j],
        dL/ddmin_b  = -w [dmin_b < 0],
        dL/dqd_jb   = 2 length qd_jb + 2 energy dt^2 qd_jb tau_jb^2   (direct),
        dL/dqdd_jb  = 2 smooth qdd_jb                                 (direct)
    (a kink takes the zero one-sided derivative).  tau, qd, qdd [d][B],
    dmin [B], limits [d].  Returns cost [B], g_tau [d][B], g_dmin [B] and,
    when qd / qdd are given, g_qd, g_qdd [d][B], all float64."""
    tau = np.asarray(tau, np.float64)
    dmin = np.asarray(dmin, np.float64)
    lo = np.asarray(tau_lo, np.float64)[:, None]
    hi = np.asarray(tau_hi, np.float64)[:, None]
    over = np.maximum(0.0, tau - hi)
    under = np.maximum(0.0, lo - tau)
    cost = (over + under).sum(axis=0) + w_coll * np.maximum(0.0, -dmin)
    g_tau = (tau > hi).astype(np.float64) - (tau < lo).astype(np.float64)
    g_dmin = -w_coll * (dmin < 0).astype(np.float64)
    if qd is None and qdd is None:
        return cost, g_tau, g_dmin
    qd = np.zeros_like(tau) if qd is None else np.asarray(qd, np.float64)
    qdd = np.zeros_like(tau) if qdd is None else np.asarray(qdd, np.float64)
    e = energy * dt * dt
    cost = cost + smooth * (qdd ** 2).sum(axis=0) + length * (qd ** 2).sum(axis=0) \
        + e * ((qd * tau) ** 2).sum(axis=0)
    g_tau = g_tau + 2.0 * e * qd ** 2 * tau
    g_qd = 2.0 * length * qd + 2.0 * e * qd * tau ** 2
    g_qdd = 2.0 * smooth * qdd
    return cost, g_tau, g_dmin, g_qd, g_qdd


def fext_gradient(robot, q, qd, qdd, fext, g_tau):
    """d<g_tau, tau>/d f_ext [B][n][6]: tau is affine in the external forces
    (f_k = I a + v x* I v - f_ext,k, link coordinates, moment then force), so
    each component is <g_tau, tau(f_ext + e) - tau(f_ext)> for a unit e."""
    r = robot
    d = r.dof
    q = np.asarray(q, np.float64)
    B = q.shape[1]
    fe = np.zeros((B, r.n, 6)) if fext is None else np.asarray(fext, np.float64)
    base = evaluate(r, q, qd, qdd, fext=fe, want=("tau",))["tau"]
    gt = np.asarray(g_tau, np.float64)
    g = np.zeros((B, r.n, 6))
    for k in range(r.n):
        for i in range(6):
            f2 = fe.copy()
            f2[:, k, i] += 1.0
            t2 = evaluate(r, q, qd, qdd, fext=f2, want=("tau",))["tau"]
            g[:, k, i] = ((t2 - base) * gt).sum(axis=0)
    return g


def kinematics(robot, q, targets, nthreads: int = 0):
    """Jacobians of the target links and the centre of mass by dual-number
    differentiation of the forward kinematics.  q [d][B].  Returns
    J [B][nt][6][d] (rows: world origin velocity, then angular velocity),
    com [B][3], Jcom [B][3][d]."""
    orob = robot if isinstance(robot, OracleRobot) else OracleRobot(robot)
    r = orob.robot
    d = r.dof
    qc = _cm(q, d)
    B = qc.shape[0]
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    J = np.zeros((B, len(tg), 6, d))
    com = np.zeros((B, 3))
    Jc = np.zeros((B, 3, d))
    rc = lib().or_kinematics(C.byref(orob.s), B, _ptr(qc), len(tg), _ptr(tg), _ptr(J), _ptr(com),
                             _ptr(Jc), nthreads)
    if rc != 0:
        raise ValueError("or_kinematics: target out of range")
    return J, com, Jc


def pair_hinge(robot, q, eta: float, w: float):
    """All-pairs summed self-collision hinge with activation distance eta:
        cost_b = w sum_p max(0, eta - d_p),  d_p = |c_i - c_j| - r_i - r_j
    over every masked pair p = (i, j), and its gradient with respect to the
    sphere centres: a pair with d_p < eta adds -w u to dcost/dc_i and +w u to
    dcost/dc_j, u = (c_i - c_j) / |c_i - c_j| (a pair exactly at eta, or with
    coincident centres, adds nothing).  q [d][B].  Returns cost [B] and
    g_sph [B][S][3] in float64."""
    r = robot
    c = evaluate(r, q, want=("sph",))["sph"]            # [B][S][3]
    P = np.asarray(r.pairs, dtype=np.int64).reshape(-1, 2)
    rad = np.asarray(r.sph_r, dtype=np.float64)
    diff = c[:, P[:, 0]] - c[:, P[:, 1]]                  # [B][P][3]
    nrm = np.sqrt((diff * diff).sum(axis=2))
    d = nrm - rad[P[:, 0]] - rad[P[:, 1]]
    act = d < eta
    cost = w * np.where(act, eta - d, 0.0).sum(axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        u = np.where(nrm[..., None] > 0, diff / nrm[..., None], 0.0)
    gu = w * u * act[..., None]
    g = np.zeros_like(c)
    for k in range(P.shape[0]):  # plain accumulation, pair by pair
        g[:, P[k, 0]] -= gu[:, k]
        g[:, P[k, 1]] += gu[:, k]
    return cost, g


def trajopt_value(robot, U, T: int, dt: float, tau_lo, tau_hi, w_coll, smooth=0.0,
                  length=0.0, energy=0.0, eta=None):
    """Total cost L(U) = sum_b cost_b over every sample of every trajectory:
    B-spline states -> whole-body evaluation -> cost (the energy term uses
    the sample spacing of the B-spline, dt (K-3) / (T-1)).  The collision
    term is w_coll max(0, -d_min) on the worst pair, or with an activation
    distance eta the summed hinge w_coll sum_p max(0, eta - d_p) over every
    masked pair (pair_hinge)."""
    q, qd, qdd = bspline(U, T, dt)
    ev = evaluate(robot, q, qd, qdd, want=("dmin", "tau"))
    K = np.asarray(U).shape[2]
    dmin = ev["dmin"] if eta is None else np.ones_like(ev["dmin"])  # hinge term apart
    cost = trajopt_cost(ev["tau"], dmin, tau_lo, tau_hi, w_coll, qd, qdd, smooth, length,
                        energy, dt * (K - 3) / (T - 1))[0]
    if eta is not None:
        cost = cost + pair_hinge(robot, q, eta, w_coll)[0]
    return float(cost.sum()), ev


def trajopt_gradient(robot, U, T: int, dt: float, tau_lo, tau_hi, w_coll, smooth=0.0,
                     length=0.0, energy=0.0, eta=None):
    """dL/dU by the chain of the pieces above: cost gradients -> VJP of the
    whole-body evaluation (dual numbers) plus the cost's direct qd / qdd
    gradients -> VJP of the B-spline.  With eta the collision term is the
    summed hinge, whose sphere-centre gradient enters the whole-body VJP.
    Returns (Ubar [n_traj][d][K], per-configuration cost [B], evaluation
    dict)."""
    U = np.asarray(U, np.float64)
    n_traj, d, K = U.shape
    q, qd, qdd = bspline(U, T, dt)
    ev = evaluate(robot, q, qd, qdd, want=("dmin", "tau"))
    dmin = ev["dmin"] if eta is None else np.ones_like(ev["dmin"])
    cost, g_tau, g_dmin, d_qd, d_qdd = trajopt_cost(ev["tau"], dmin, tau_lo, tau_hi,
                                                    w_coll, qd, qdd, smooth, length, energy,
                                                    dt * (K - 3) / (T - 1))
    if eta is None:
        gq, gqd, gqdd = gradient(robot, q, qd, qdd, g_dmin=g_dmin, g_tau=g_tau)
    else:
        hc, g_sph = pair_hinge(robot, q, eta, w_coll)
        cost = cost + hc
        gq, gqd, gqdd = gradient(robot, q, qd, qdd, g_sph=g_sph, g_tau=g_tau)
    return bspline_vjp(gq, gqd + d_qd, gqdd + d_qdd, n_traj, K, T, dt), cost, ev


def max_threads() -> int:
    return int(lib().or_max_threads())
