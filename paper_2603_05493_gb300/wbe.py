"""Python binding of the whole-body evaluation library.

Every computation runs in libwbe.so's CUDA kernels; this module only builds
the C descriptors, hands device pointers of torch tensors and the current
stream across the C ABI, and wraps the pair of calls in a
torch.autograd.Function.

Tensor layouts (float32 unless noted, on the robot's CUDA device):
  q, qd, qdd, tau, grads   (d, B)     joint-major
  link_pose                (B, n, 12) world R (row-major) then p
  sphere                   (B, S, 3)
  d_min                    (B,)
  worst                    (B,) int32
  pair_bits                (B, ceil(P/32)) int32 holding uint32 bit words
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


def _arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


@dataclass
class Tune:
    """Kernel choice and launch shape (zeros = automatic)."""
    kernel: int = L.WB_KERNEL_AUTO
    lanes_per_config: int = 0
    configs_per_block: int = 0
    blocks_per_sm: int = 0

    def c(self):
        return L.wb_tune(self.kernel, self.lanes_per_config, self.configs_per_block,
                         self.blocks_per_sm)


PLAIN = Tune(kernel=L.WB_KERNEL_PLAIN)
FUSED = Tune(kernel=L.WB_KERNEL_FUSED)
TREE = Tune(kernel=L.WB_KERNEL_TREE)
TREE_NOCULL = Tune(kernel=L.WB_KERNEL_TREE_NOCULL)


def _inertial_struct(keep, mass, com, inertia, pm_link=None, pm_mass=None, pm_pos=None):
    def k(a, dt):
        a = _arr(a, dt)
        keep.append(a)
        return a.ctypes.data
    npm = 0 if pm_link is None else len(pm_link)
    return L.wb_inertial(k(mass, np.float64), k(com, np.float64), k(inertia, np.float64), npm,
                         k(pm_link, np.int32) if npm else None,
                         k(pm_mass, np.float64) if npm else None,
                         k(pm_pos, np.float64) if npm else None)


def descriptors(desc, keep):
    """C descriptor structs for a robot description (see Robot); the numpy
    buffers they point to are appended to `keep`."""
    def k(a, dt):
        a = _arr(a, dt)
        keep.append(a)
        return a.ctypes.data

    n = len(desc.parent)
    tree = L.wb_tree(n, k(desc.parent, np.int32), k(desc.jtype, np.int32),
                     k(desc.axis, np.float64), k(desc.T_fixed, np.float64),
                     k(desc.jidx, np.int32), k(desc.mimic_mult, np.float64),
                     k(desc.mimic_off, np.float64), k(desc.gravity, np.float64))
    S = len(desc.sph_r)
    sph = L.wb_spheres(S, k(desc.sph_link, np.int32), k(desc.sph_c, np.float64),
                       k(desc.sph_r, np.float64))
    pr = _arr(desc.pairs, np.int32).reshape(-1, 2)
    keep.append(pr)
    pairs = L.wb_pairs(pr.shape[0], pr.ctypes.data if pr.size else None, None)
    pm = getattr(desc, "pm_link", None)
    inert = _inertial_struct(keep, desc.mass, desc.com, desc.Icom,
                             pm if pm is not None and len(pm) else None,
                             getattr(desc, "pm_mass", None), getattr(desc, "pm_pos", None))
    return tree, sph, pairs, inert


def plan_info(desc):
    """Validate and plan a robot on the host only (no GPU needed).  Returns
    (info dict, pair-schedule rounds for 4/8/16/32 lanes per configuration)."""
    lib = L.load()
    keep = []
    tree, sph, pairs, inert = descriptors(desc, keep)
    info = L.wb_robot_info()
    rounds = (C.c_int32 * 4)()
    L.check(lib.wb_plan_info(C.byref(tree), C.byref(sph), C.byref(pairs), C.byref(inert),
                             C.byref(info), rounds), "wb_plan_info")
    d = {f: getattr(info, f) for f, _ in L.wb_robot_info._fields_}
    return d, list(rounds)


class Robot:
    """A robot loaded into libwbe on one CUDA device.

    `desc` is any object with the descriptor arrays: parent, jtype, axis,
    T_fixed, jidx, mimic_mult, mimic_off, gravity, sph_link, sph_c, sph_r,
    pairs (P, 2), mass, com, Icom and optionally pm_link, pm_mass, pm_pos
    (payload point masses)."""

    def __init__(self, desc, device=None):
        self.lib = L.load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", int(device))
        keep = []
        tree, sph, pairs, inert = descriptors(desc, keep)
        h = C.c_void_p()
        L.check(self.lib.wb_load_robot(C.byref(tree), C.byref(sph), C.byref(pairs),
                                       C.byref(inert), int(self.device.index), C.byref(h)),
                "wb_load_robot")
        self.handle = h
        info = L.wb_robot_info()
        L.check(self.lib.wb_robot_info_get(self.handle, C.byref(info)), "wb_robot_info_get")
        self.n, self.dof, self.S, self.P = info.n_links, info.dof, info.n_spheres, info.n_pairs
        self.n_levels = info.n_levels
        self.max_level_width = info.max_level_width
        self.n_pair_blocks = info.n_pair_blocks

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.lib.wb_free_robot(h)
            self.handle = None

    @property
    def pair_words(self) -> int:
        return (self.P + 31) // 32

    def set_inertials(self, mass, com, inertia, pm_link=None, pm_mass=None, pm_pos=None,
                      stream=None):
        keep = []
        inert = _inertial_struct(keep, mass, com, inertia, pm_link, pm_mass, pm_pos)
        L.check(self.lib.wb_set_inertials(self.handle, C.byref(inert), _stream(stream)),
                "wb_set_inertials")

    def autotune(self, B):
        """Time the kernel families / launch shapes on this robot for batch B;
        returns (forward Tune, backward Tune, forward ms, backward ms)."""
        f, b = L.wb_tune(), L.wb_tune()
        fm, bm = C.c_float(), C.c_float()
        L.check(self.lib.wb_autotune(self.handle, int(B), C.byref(f), C.byref(b), C.byref(fm),
                                     C.byref(bm)), "wb_autotune")
        mk = lambda t: Tune(t.kernel, t.lanes_per_config, t.configs_per_block, t.blocks_per_sm)
        return mk(f), mk(b), fm.value, bm.value

    def autotune_spline(self, n_traj: int, K: int, T: int, dt: float, w_coll: float = 1.0,
                        smooth: float = 0.0, length: float = 0.0, energy: float = 0.0,
                        dt_cost: float = 1.0):
        """Time the sweep shapes of the control-point path (eval_spline's
        forward sweep and eval_backward_spline_cost with these cost weights)
        for n_traj trajectories of T samples from K control points
        (wb_autotune_spline); returns (forward Tune, backward Tune, forward
        ms, backward ms)."""
        f, b = L.wb_tune(), L.wb_tune()
        fm, bm = C.c_float(), C.c_float()
        w = L.wb_cost_weights(float(w_coll), float(smooth), float(length), float(energy),
                              float(dt_cost))
        L.check(self.lib.wb_autotune_spline(self.handle, int(n_traj), int(K), int(T), float(dt),
                                            C.byref(w), C.byref(f), C.byref(b), C.byref(fm),
                                            C.byref(bm)), "wb_autotune_spline")
        mk = lambda t: Tune(t.kernel, t.lanes_per_config, t.configs_per_block, t.blocks_per_sm)
        return mk(f), mk(b), fm.value, bm.value

    # ------------------------------------------------------------------
    def empty_outputs(self, B, pose=True, sphere=True, dmin=True, tau=True, bits=False):
        dev = self.device
        f = dict(device=dev, dtype=torch.float32)
        return {
            "pose": torch.empty((B, self.n, 12), **f) if pose else None,
            "sphere": torch.empty((B, self.S, 3), **f) if sphere else None,
            "dmin": torch.empty((B,), **f) if dmin else None,
            "worst": torch.empty((B,), device=dev, dtype=torch.int32) if dmin else None,
            "tau": torch.empty((self.dof, B), **f) if tau else None,
            "bits": torch.empty((B, max(self.pair_words, 1)), device=dev, dtype=torch.int32)
            if bits else None,
        }

    def eval(self, q, qd=None, qdd=None, *, pose=True, sphere=True, dmin=True, tau=True,
             bits=False, tune: Tune | None = None, out=None, f_ext=None, stream=None):
        """Forward whole-body evaluation; returns a dict of output tensors.
        f_ext: optional external link wrenches [B][n][6] (wb_eval_ext)."""
        B = q.shape[1]
        o = out if out is not None else self.empty_outputs(B, pose, sphere, dmin, tau, bits)
        t = (tune or Tune()).c()
        L.check(self.lib.wb_eval_ext(self.handle, B, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(f_ext),
                                     _ptr(o["pose"]), _ptr(o["sphere"]), _ptr(o["dmin"]),
                                     _ptr(o["worst"]), _ptr(o["tau"]), _ptr(o["bits"]),
                                     C.byref(t), _stream(stream)),
                "wb_eval")
        return o

    def self_collision(self, link_pose, *, sphere=True, dmin=True, bits=False, diff=False,
                       out=None, tune: Tune | None = None, stream=None):
        """Spheres and the pair map-reduce from given world link poses
        (B, n, 12); returns a dict with sphere, dmin, worst, bits and, with
        diff=True (or a "diff" tensor in `out`), the worst pair's centre
        difference (B, 3) for eval_backward's worst_diff
        (wb_self_collision_dir).  tune: TREE (default, culled blocks) or
        Tune(kernel=TREE_NOCULL)."""
        B = link_pose.shape[0]
        o = out if out is not None else self.empty_outputs(B, pose=False, sphere=sphere,
                                                           dmin=dmin, tau=False, bits=bits)
        if out is None and diff:
            o["diff"] = torch.empty((B, 3), device=self.device, dtype=torch.float32)
        t = (tune or Tune()).c()
        L.check(self.lib.wb_self_collision_dir(self.handle, B, _ptr(link_pose),
                                               _ptr(o.get("sphere")), _ptr(o.get("dmin")),
                                               _ptr(o.get("worst")), _ptr(o.get("diff")),
                                               _ptr(o.get("bits")), C.byref(t), _stream(stream)),
                "wb_self_collision")
        return o

    def kinematics(self, link_pose, targets=(), *, jac=None, com=True, jac_com=True,
                   stream=None):
        """Jacobians of the target links [B][nt][6][d], centre of mass [B][3]
        and its Jacobian [B][3][d] from world link poses (wb_kinematics);
        pass False to skip an output."""
        B = link_pose.shape[0]
        f = dict(device=link_pose.device, dtype=torch.float32)
        tg = (C.c_int32 * max(len(targets), 1))(*[int(t) for t in targets])
        if jac is None and len(targets):
            jac = torch.empty((B, len(targets), 6, self.dof), **f)
        if com is True:
            com = torch.empty((B, 3), **f)
        elif com is False:
            com = None
        if jac_com is True:
            jac_com = torch.empty((B, 3, self.dof), **f)
        elif jac_com is False:
            jac_com = None
        L.check(self.lib.wb_kinematics(self.handle, B, _ptr(link_pose), len(targets), tg,
                                       _ptr(jac), _ptr(com), _ptr(jac_com), _stream(stream)),
                "wb_kinematics")
        return jac, com, jac_com

    def self_collision_hinge(self, link_pose, eta: float, w: float = 1.0, *, cost=None,
                             g_sphere=None, want_grad=True, stream=None):
        """All-pairs summed collision hinge w * sum max(0, eta - d) per
        configuration and its sphere-centre gradient (wb_self_collision_hinge);
        returns (cost [B], g_sphere [B][S][3] or None)."""
        B = link_pose.shape[0]
        f = dict(device=link_pose.device, dtype=torch.float32)
        cost = cost if cost is not None else torch.empty((B,), **f)
        if g_sphere is None and want_grad:
            g_sphere = torch.empty((B, self.S, 3), **f)
        L.check(self.lib.wb_self_collision_hinge(self.handle, B, _ptr(link_pose), float(eta),
                                                 float(w), _ptr(cost), _ptr(g_sphere),
                                                 _stream(stream)),
                "wb_self_collision_hinge")
        return cost, g_sphere

    def eval_backward(self, q, qd, qdd, worst=None, g_pose=None, g_sphere=None, g_dmin=None,
                      g_tau=None, *, tune: Tune | None = None, out=None, f_ext=None,
                      g_fext=None, worst_diff=None, stream=None):
        """Gradient of <g_pose,pose> + <g_sphere,sphere> + g_dmin.d_min +
        <g_tau,tau> w.r.t. (q, qd, qdd); with f_ext given (the forward's
        external wrenches) and a g_fext buffer [B][n][6], also w.r.t. f_ext;
        worst_diff: the pair stage's centre difference of the worst pair (B, 3)
        (wb_eval_backward_dir)."""
        B = q.shape[1]
        if out is None:
            out = tuple(torch.empty((self.dof, B), device=self.device, dtype=torch.float32)
                        for _ in range(3))
        gq, gqd, gqdd = out
        t = (tune or Tune()).c()
        L.check(self.lib.wb_eval_backward_dir(self.handle, B, _ptr(q), _ptr(qd), _ptr(qdd),
                                              _ptr(f_ext), _ptr(worst), _ptr(worst_diff),
                                              _ptr(g_pose), _ptr(g_sphere), _ptr(g_dmin),
                                              _ptr(g_tau), _ptr(gq), _ptr(gqd), _ptr(gqdd),
                                              _ptr(g_fext), C.byref(t), _stream(stream)),
                "wb_eval_backward")
        return gq, gqd, gqdd

    def _spline(self, U, T: int, dt: float):
        n_traj, d, K = U.shape
        return L.wb_spline(U.data_ptr(), int(n_traj), int(K), int(T), float(dt)), int(n_traj) * int(T)

    def eval_spline(self, U, T: int, dt: float, *, pose=True, sphere=True, dmin=True, tau=True,
                    tune: Tune | None = None, out=None, stream=None):
        """Forward evaluation with the joint states evaluated from B-spline
        control points U [n_traj][d][K] inside the sweep (wb_eval_spline);
        returns the output dict of eval (no pair bits)."""
        sp, B = self._spline(U, T, dt)
        o = out if out is not None else self.empty_outputs(B, pose, sphere, dmin, tau, False)
        t = (tune or Tune()).c()
        L.check(self.lib.wb_eval_spline(self.handle, C.byref(sp), _ptr(o.get("pose")),
                                        _ptr(o.get("sphere")), _ptr(o.get("dmin")),
                                        _ptr(o.get("worst")), _ptr(o.get("tau")), C.byref(t),
                                        _stream(stream)), "wb_eval_spline")
        return o

    def eval_backward_spline_cost(self, U, T: int, dt: float, tau, tau_lo, tau_hi,
                                  w_coll: float, smooth: float = 0.0, length: float = 0.0,
                                  energy: float = 0.0, dt_cost: float = 1.0, *, d_min=None,
                                  worst=None, g_pose=None, g_sphere=None, cost=None,
                                  want_cost: bool = True, tune: Tune | None = None, out=None,
                                  worst_diff=None, stream=None):
        """eval_backward_cost with the joint states evaluated from control
        points (wb_eval_backward_spline_cost_dir).  dt_cost is the energy
        term's dt; worst_diff: the pair stage's worst-pair centre difference.
        Returns (gq, gqd, gqdd, cost)."""
        sp, B = self._spline(U, T, dt)
        if out is None:
            out = tuple(torch.empty((self.dof, B), device=self.device, dtype=torch.float32)
                        for _ in range(3))
        gq, gqd, gqdd = out
        if cost is None and want_cost:
            cost = torch.empty((B,), device=self.device, dtype=torch.float32)
        w = L.wb_cost_weights(float(w_coll), float(smooth), float(length), float(energy),
                              float(dt_cost))
        t = (tune or Tune()).c()
        L.check(self.lib.wb_eval_backward_spline_cost_dir(
            self.handle, C.byref(sp), _ptr(worst), _ptr(worst_diff), _ptr(g_pose),
            _ptr(g_sphere), _ptr(tau), _ptr(d_min), _ptr(tau_lo), _ptr(tau_hi), C.byref(w),
            _ptr(cost), _ptr(gq), _ptr(gqd), _ptr(gqdd), C.byref(t), _stream(stream)),
            "wb_eval_backward_spline_cost")
        return gq, gqd, gqdd, cost

    def eval_backward_cost(self, q, qd, qdd, tau, tau_lo, tau_hi, w_coll: float,
                           smooth: float = 0.0, length: float = 0.0, energy: float = 0.0,
                           dt: float = 1.0, *, d_min=None, worst=None, g_pose=None,
                           g_sphere=None, cost=None, want_cost: bool = True,
                           tune: Tune | None = None, out=None, worst_diff=None, stream=None):
        """The trajectory cost folded into the backward sweep
        (wb_eval_backward_cost_dir; worst_diff as eval_backward takes it):
        total gradients (gq, gqd, gqdd) of the
        per-configuration cost (torque hinges, worst-pair hinge when d_min
        is given, smooth / length / energy terms) plus <g_pose, poses> +
        <g_sphere, centres>, and the cost [B].  Returns (gq, gqd, gqdd,
        cost)."""
        B = q.shape[1]
        if out is None:
            out = tuple(torch.empty((self.dof, B), device=self.device, dtype=torch.float32)
                        for _ in range(3))
        gq, gqd, gqdd = out
        if cost is None and want_cost:
            cost = torch.empty((B,), device=self.device, dtype=torch.float32)
        w = L.wb_cost_weights(float(w_coll), float(smooth), float(length), float(energy),
                              float(dt))
        t = (tune or Tune()).c()
        L.check(self.lib.wb_eval_backward_cost_dir(self.handle, B, _ptr(q), _ptr(qd),
                                                   _ptr(qdd), _ptr(worst), _ptr(worst_diff),
                                                   _ptr(g_pose), _ptr(g_sphere), _ptr(tau),
                                                   _ptr(d_min), _ptr(tau_lo), _ptr(tau_hi),
                                                   C.byref(w), _ptr(cost), _ptr(gq), _ptr(gqd),
                                                   _ptr(gqdd), C.byref(t), _stream(stream)),
                "wb_eval_backward_cost")
        return gq, gqd, gqdd, cost


class Batch:
    """An uneven batch: problems (robot index, horizon) over several loaded
    robots, evaluated by one persistent launch per pass.  Packed arrays are
    flat float32 / int32 tensors of the lengths in `sizes`; problem p's slices
    start at the offsets in `offsets` (see include/wbe.h)."""

    def __init__(self, robots, problems):
        self.lib = L.load()
        self.robots = list(robots)
        self.device = self.robots[0].device
        arr = (C.c_void_p * len(self.robots))(*[r.handle.value for r in self.robots])
        probs = (L.wb_problem * len(problems))(*[L.wb_problem(int(a), int(h))
                                                 for a, h in problems])
        h = C.c_void_p()
        L.check(self.lib.wb_batch_create(arr, len(self.robots), probs, len(problems),
                                         C.byref(h)), "wb_batch_create")
        self.handle = h
        sz = L.wb_batch_sizes()
        L.check(self.lib.wb_batch_sizes_get(self.handle, C.byref(sz)), "wb_batch_sizes_get")
        self.sizes = {f: getattr(sz, f) for f, _ in L.wb_batch_sizes._fields_}
        n = len(problems)
        offs = [np.zeros(n, np.int64) for _ in range(4)]
        L.check(self.lib.wb_batch_offsets(self.handle, *[o.ctypes.data for o in offs]),
                "wb_batch_offsets")
        self.offsets = {"joint": offs[0], "pose": offs[1], "sphere": offs[2], "config": offs[3]}
        self.problems = [(int(a), int(h)) for a, h in problems]

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            self.lib.wb_free_batch(h)
            self.handle = None

    def empty(self, kind, dtype=torch.float32):
        n = {"joint": "joint_elems", "pose": "pose_elems", "sphere": "sphere_elems",
             "config": "configs"}[kind]
        return torch.empty(max(self.sizes[n], 1), device=self.device, dtype=dtype)

    def pack_joint(self, per_problem):
        """Concatenate per-problem [d][H] arrays into the packed joint layout."""
        out = self.empty("joint")
        for p, x in enumerate(per_problem):
            o = int(self.offsets["joint"][p])
            out[o:o + x.numel()] = torch.as_tensor(x, device=self.device).reshape(-1)
        return out

    def view(self, packed, kind, p, shape):
        o = int(self.offsets[kind][p])
        n = int(np.prod(shape))
        return packed[o:o + n].view(*shape)

    def set_tune(self, fwd_threads=0, bwd_threads=0, pair_warps=0, fwd_segments=None,
                 bwd_segments=None):
        """Launch choices of the batch's passes (wb_batch_set_tune): sweep
        threads per block, pair warps per block, and per robot 1 or 2 sweep
        segments for each pass (None = the defaults)."""
        t = L.wb_batch_tune(int(fwd_threads), int(bwd_threads), int(pair_warps))
        segs = [None if x is None else np.ascontiguousarray(x, dtype=np.int32)
                for x in (fwd_segments, bwd_segments)]
        L.check(self.lib.wb_batch_set_tune(self.handle, C.byref(t),
                                           *[None if x is None else x.ctypes.data for x in segs]),
                "wb_batch_set_tune")

    def get_tune(self):
        """(wb_batch_tune as a dict, forward segments, backward segments)."""
        t = L.wb_batch_tune()
        f = np.zeros(len(self.robots), np.int32)
        b = np.zeros(len(self.robots), np.int32)
        L.check(self.lib.wb_batch_get_tune(self.handle, C.byref(t), f.ctypes.data, b.ctypes.data),
                "wb_batch_get_tune")
        return {k: getattr(t, k) for k, _ in L.wb_batch_tune._fields_}, f.tolist(), b.tolist()

    def autotune(self):
        """Time the batch's launch choices and keep the fastest
        (wb_batch_autotune); returns (tune dict, forward segments, backward
        segments, forward ms, backward ms)."""
        t = L.wb_batch_tune()
        f = np.zeros(len(self.robots), np.int32)
        b = np.zeros(len(self.robots), np.int32)
        fm, bm = C.c_float(), C.c_float()
        L.check(self.lib.wb_batch_autotune(self.handle, C.byref(t), f.ctypes.data, b.ctypes.data,
                                           C.byref(fm), C.byref(bm)), "wb_batch_autotune")
        return ({k: getattr(t, k) for k, _ in L.wb_batch_tune._fields_}, f.tolist(), b.tolist(),
                fm.value, bm.value)

    def eval(self, q, qd, qdd, pose, sphere=None, dmin=None, worst=None, tau=None, stream=None):
        L.check(self.lib.wb_batch_eval(self.handle, _ptr(q), _ptr(qd), _ptr(qdd), _ptr(pose),
                                       _ptr(sphere), _ptr(dmin), _ptr(worst), _ptr(tau),
                                       _stream(stream)), "wb_batch_eval")

    def eval_backward(self, q, qd, qdd, worst, g_pose, g_sphere, g_dmin, g_tau, gq, gqd, gqdd,
                      stream=None):
        L.check(self.lib.wb_batch_eval_backward(self.handle, _ptr(q), _ptr(qd), _ptr(qdd),
                                                _ptr(worst), _ptr(g_pose), _ptr(g_sphere),
                                                _ptr(g_dmin), _ptr(g_tau), _ptr(gq), _ptr(gqd),
                                                _ptr(gqdd), _stream(stream)),
                "wb_batch_eval_backward")


def bspline_eval(U, T: int, dt: float, q=None, qd=None, qdd=None, stream=None, start=None,
                 end_static: bool = False):
    """Joint states [d][n_traj*T] from B-spline control points U
    [n_traj][d][K] (wb_bspline_eval); allocates the outputs it is not given.
    With ``start`` [n_traj][d][3] (theta_0, thetadot_0, thetaddot_0) the
    ghost knots of that start state come first, and ``end_static`` repeats
    the last control point for a static goal (wb_bspline_eval_bc)."""
    lib = L.load()
    n_traj, d, K = U.shape
    B = n_traj * T
    mk = lambda t: t if t is not None else torch.empty((d, B), device=U.device)  # noqa: E731
    q, qd, qdd = mk(q), mk(qd), mk(qdd)
    if start is None and not end_static:
        L.check(lib.wb_bspline_eval(n_traj, d, K, int(T), float(dt), _ptr(U), _ptr(q), _ptr(qd),
                                    _ptr(qdd), _stream(stream)), "wb_bspline_eval")
    else:
        L.check(lib.wb_bspline_eval_bc(n_traj, d, K, int(T), float(dt), _ptr(U), _ptr(start),
                                       1 if end_static else 0, _ptr(q), _ptr(qd), _ptr(qdd),
                                       _stream(stream)), "wb_bspline_eval_bc")
    return q, qd, qdd


def bspline_backward_bc(gq, gqd, gqdd, n_traj: int, K: int, T: int, dt: float,
                        has_start: bool = False, end_static: bool = False, gU=None,
                        g_start=None, want_start: bool = True, gqd_add=None, gqdd_add=None,
                        stream=None):
    """Gradients through bspline_eval with boundary conditions
    (wb_bspline_backward_bc): the control-point gradient [n_traj][d][K] and,
    with a start state (and want_start), the start-state gradient
    [n_traj][d][3].  Returns (gU, g_start)."""
    lib = L.load()
    ref = next(t for t in (gq, gqd, gqdd, gqd_add, gqdd_add) if t is not None)
    d = ref.shape[0]
    if gU is None:
        gU = torch.empty((n_traj, d, K), device=ref.device)
    if g_start is None and has_start and want_start:
        g_start = torch.empty((n_traj, d, 3), device=ref.device)
    L.check(lib.wb_bspline_backward_bc(n_traj, d, K, int(T), float(dt), 1 if has_start else 0,
                                       1 if end_static else 0, _ptr(gq), _ptr(gqd), _ptr(gqdd),
                                       _ptr(gqd_add), _ptr(gqdd_add), _ptr(gU), _ptr(g_start),
                                       _stream(stream)), "wb_bspline_backward_bc")
    return gU, g_start


def bspline_backward(gq, gqd, gqdd, n_traj: int, K: int, T: int, dt: float, gU=None,
                     stream=None, gqd_add=None, gqdd_add=None):
    """Control-point gradient [n_traj][d][K] from upstream gradients on the
    states (wb_bspline_backward; any of gq, gqd, gqdd may be None).  With
    gqd_add / gqdd_add (wb_bspline_backward_ext) those add to gqd / gqdd."""
    lib = L.load()
    ref = next(t for t in (gq, gqd, gqdd, gqd_add, gqdd_add) if t is not None)
    d = ref.shape[0]
    if gU is None:
        gU = torch.empty((n_traj, d, K), device=ref.device)
    if gqd_add is None and gqdd_add is None:
        L.check(lib.wb_bspline_backward(n_traj, d, K, int(T), float(dt), _ptr(gq), _ptr(gqd),
                                        _ptr(gqdd), _ptr(gU), _stream(stream)),
                "wb_bspline_backward")
    else:
        L.check(lib.wb_bspline_backward_ext(n_traj, d, K, int(T), float(dt), _ptr(gq),
                                            _ptr(gqd), _ptr(gqdd), _ptr(gqd_add),
                                            _ptr(gqdd_add), _ptr(gU), _stream(stream)),
                "wb_bspline_backward_ext")
    return gU


def trajopt_cost(tau, d_min, tau_lo, tau_hi, w_coll: float, cost=None, g_tau=None, g_dmin=None,
                 stream=None):
    """Per-configuration cost and upstream gradients (wb_trajopt_cost);
    allocates the outputs it is not given.  Returns (cost, g_tau, g_dmin)."""
    lib = L.load()
    ref = tau if tau is not None else d_min
    d, B = tau.shape if tau is not None else (0, d_min.shape[0])
    cost = cost if cost is not None else torch.empty((B,), device=ref.device)
    if g_tau is None and tau is not None:
        g_tau = torch.empty((d, B), device=ref.device)
    if g_dmin is None and d_min is not None:
        g_dmin = torch.empty((B,), device=ref.device)
    L.check(lib.wb_trajopt_cost(B, d, _ptr(tau), _ptr(d_min), _ptr(tau_lo), _ptr(tau_hi),
                                float(w_coll), _ptr(cost), _ptr(g_tau), _ptr(g_dmin),
                                _stream(stream)), "wb_trajopt_cost")
    return cost, g_tau, g_dmin


def trajopt_cost_ext(tau, d_min, qd, qdd, tau_lo, tau_hi, w_coll: float, smooth: float = 0.0,
                     length: float = 0.0, energy: float = 0.0, dt: float = 1.0, out=None,
                     stream=None):
    """The cost with its motion terms (wb_trajopt_cost_ext): smooth |qdd|^2,
    length |qd|^2 and energy sum_j (qd_j tau_j dt)^2 on top of the hinges.
    ``out`` may hold preallocated (cost, g_tau, g_dmin, g_qd, g_qdd); the
    ones missing are allocated.  Returns (cost, g_tau, g_dmin, g_qd, g_qdd)."""
    lib = L.load()
    ref = next(t for t in (tau, qd, qdd, d_min) if t is not None)
    d, B = ref.shape if ref.dim() == 2 else (0, ref.shape[0])
    cost, g_tau, g_dmin, g_qd, g_qdd = out if out is not None else (None,) * 5
    mk = lambda t, src, shape: t if t is not None or src is None else \
        torch.empty(shape, device=ref.device)  # noqa: E731
    cost = mk(cost, ref, (B,))
    g_tau, g_dmin = mk(g_tau, tau, (d, B)), mk(g_dmin, d_min, (B,))
    g_qd, g_qdd = mk(g_qd, qd, (d, B)), mk(g_qdd, qdd, (d, B))
    w = L.wb_cost_weights(float(w_coll), float(smooth), float(length), float(energy), float(dt))
    L.check(lib.wb_trajopt_cost_ext(B, d, _ptr(tau), _ptr(d_min), _ptr(qd), _ptr(qdd),
                                    _ptr(tau_lo), _ptr(tau_hi), C.byref(w), _ptr(cost),
                                    _ptr(g_tau), _ptr(g_dmin), _ptr(g_qd), _ptr(g_qdd),
                                    _stream(stream)), "wb_trajopt_cost_ext")
    return cost, g_tau, g_dmin, g_qd, g_qdd


def batch_eval_noalloc(robots, problems, q, qd, qdd, pose, sphere=None, dmin=None, worst=None,
                       tau=None, stream=None):
    """wb_batch_eval_noalloc: forward evaluation of an uneven batch without any
    device allocation, for callers whose problem mix changes every call and
    who cannot afford (or are not allowed) to allocate device memory per call.
    Buffers are packed as for `Batch` built from the same problems; all of
    them are the caller's.  Calls on one device must not overlap on the GPU
    (they share the library's scratch), and the first call on a device does a
    one-time setup (include/wbe.h)."""
    lib = L.load()
    robots = list(robots)
    arr = (C.c_void_p * len(robots))(*[r.handle.value for r in robots])
    probs = (L.wb_problem * max(len(problems), 1))(*[L.wb_problem(int(a), int(h))
                                                     for a, h in problems])
    L.check(lib.wb_batch_eval_noalloc(arr, len(robots), probs, len(problems), _ptr(q), _ptr(qd),
                                      _ptr(qdd), _ptr(pose), _ptr(sphere), _ptr(dmin),
                                      _ptr(worst), _ptr(tau), _stream(stream)),
            "wb_batch_eval_noalloc")


class StreamedStep:
    """Forward + backward over a batch whose inputs and outputs live in pinned
    host memory.  The batch is cut into chunks with their own device buffers;
    the host-to-device copies of one chunk, the kernels of another and the
    device-to-host copies of a third run on three streams, so transfers in
    both directions overlap each other and the evaluation.  Per step and
    chunk c: inputs host_in[c] = dict(q, qd, qdd [d][Bc], g_pose [Bc][n][12],
    g_sphere [Bc][S][3], g_dmin [Bc], g_tau [d][Bc]) copied in; outputs
    host_out[c] = dict(pose, sphere, dmin, worst, tau, gq, gqd, gqdd) copied
    out.  Events per chunk order consecutive steps (a chunk's inputs are not
    overwritten before its kernels ran, nor its outputs before they were
    copied out).  step() enqueues and returns; the caller's current stream
    waits for the last copy."""

    IN = ("q", "qd", "qdd", "g_pose", "g_sphere", "g_dmin", "g_tau")
    OUT = ("pose", "sphere", "dmin", "worst", "tau", "gq", "gqd", "gqdd")

    def __init__(self, robot: Robot, chunk: int, n_chunks: int, fwd_tune: Tune | None = None,
                 bwd_tune: Tune | None = None, run_streams: int = 1):
        self.rob, self.Bc, self.K = robot, int(chunk), int(n_chunks)
        self.ft, self.bt = fwd_tune or TREE, bwd_tune or TREE
        dev, d, n, S, Bc = robot.device, robot.dof, robot.n, robot.S, self.Bc
        f = dict(device=dev, dtype=torch.float32)
        self.din, self.dout = [], []
        for _ in range(self.K):
            self.din.append({"q": torch.empty((d, Bc), **f), "qd": torch.empty((d, Bc), **f),
                             "qdd": torch.empty((d, Bc), **f),
                             "g_pose": torch.empty((Bc, n, 12), **f),
                             "g_sphere": torch.empty((Bc, S, 3), **f),
                             "g_dmin": torch.empty((Bc,), **f),
                             "g_tau": torch.empty((d, Bc), **f)})
            o = robot.empty_outputs(Bc)
            o.update(gq=torch.empty((d, Bc), **f), gqd=torch.empty((d, Bc), **f),
                     gqdd=torch.empty((d, Bc), **f),
                     diff=torch.empty((Bc, 3), **f))  # the worst pair's, stays on the device
            self.dout.append(o)
        self.s_in, self.s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        # chunks alternate over run_streams compute streams, so that the kernels
        # of consecutive chunks may share the GPU
        self.s_runs = [torch.cuda.Stream(dev) for _ in range(max(1, int(run_streams)))]
        self.ev_in = [torch.cuda.Event() for _ in range(self.K)]
        self.ev_run = [torch.cuda.Event() for _ in range(self.K)]
        self.ev_out = [torch.cuda.Event() for _ in range(self.K)]

    def host_buffers(self):
        """Pinned host inputs and outputs shaped for step()."""
        hin = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in c.items()}
               for c in self.din]
        hout = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                 for k, v in c.items() if k in self.OUT and v is not None} for c in self.dout]
        return hin, hout

    def step(self, host_in, host_out):
        rob = self.rob
        for c in range(self.K):
            di, do = self.din[c], self.dout[c]
            self.s_in.wait_event(self.ev_run[c])  # the last step's kernels read di
            with torch.cuda.stream(self.s_in):
                for k in self.IN:
                    di[k].copy_(host_in[c][k], non_blocking=True)
                self.ev_in[c].record(self.s_in)
            sr = self.s_runs[c % len(self.s_runs)]
            sr.wait_event(self.ev_in[c])
            sr.wait_event(self.ev_out[c])  # the last step's copies read do
            with torch.cuda.stream(sr):
                fwd = {"pose": do["pose"], "sphere": None, "dmin": None, "worst": None,
                       "tau": do["tau"], "bits": None}  # the sweep; pairs follow
                rob.eval(di["q"], di["qd"], di["qdd"], tune=self.ft, out=fwd, stream=sr)
                rob.self_collision(do["pose"], out=do, stream=sr)
                rob.eval_backward(di["q"], di["qd"], di["qdd"], do["worst"], di["g_pose"],
                                  di["g_sphere"], di["g_dmin"], di["g_tau"], tune=self.bt,
                                  out=(do["gq"], do["gqd"], do["gqdd"]), stream=sr,
                                  worst_diff=do["diff"])
                self.ev_run[c].record(sr)
            self.s_out.wait_event(self.ev_run[c])
            with torch.cuda.stream(self.s_out):
                for k, v in host_out[c].items():
                    v.copy_(do[k], non_blocking=True)
                self.ev_out[c].record(self.s_out)
        torch.cuda.current_stream().wait_event(self.ev_out[self.K - 1])  # s_out is in order


def descriptor_hash(desc) -> str:
    """Content hash of a robot description (the autotune cache key)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("parent", "jtype", "axis", "T_fixed", "jidx", "mimic_mult", "mimic_off",
                 "gravity", "sph_link", "sph_c", "sph_r", "pairs", "mass", "com", "Icom"):
        h.update(np.ascontiguousarray(getattr(desc, name)).tobytes())
    return h.hexdigest()[:32]


def autotune_cached(robot: Robot, desc, B: int, path: str | None = None):
    """Autotune once per (robot description, GPU, batch size); results persist
    in a JSON file (default ~/.cache/wbe/autotune.json)."""
    import json
    import os
    path = path or os.path.join(os.path.expanduser("~"), ".cache", "wbe", "autotune.json")
    key = "%s|%s|%d|%d" % (descriptor_hash(desc), torch.cuda.get_device_name(robot.device), B,
                           L.load().wb_version())
    cache = {}
    if os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    if key in cache:
        e = cache[key]
        return Tune(*e["fwd"]), Tune(*e["bwd"]), e["fwd_ms"], e["bwd_ms"]
    f, b, fm, bm = robot.autotune(B)
    fields = lambda t: [t.kernel, t.lanes_per_config, t.configs_per_block,  # noqa: E731
                        t.blocks_per_sm]
    cache[key] = {"fwd": fields(f), "bwd": fields(b), "fwd_ms": fm, "bwd_ms": bm}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1)
    os.replace(tmp, path)
    return f, b, fm, bm


def _c(t):
    return None if t is None else t.contiguous()


class WholeBodyEval(torch.autograd.Function):
    """(q, qd, qdd) -> (link_pose, sphere, d_min, tau) with the hand-written
    adjoint kernel as backward.  Saves q, qd, qdd, the worst pair and its
    centre difference (3 floats a configuration), not the transforms (they
    are recomputed).  With the default or the tree kernels the forward runs
    as the sweep, then the pair stage, which also hands the backward the
    worst pair's centre difference."""

    @staticmethod
    def forward(ctx, robot: Robot, q, qd, qdd, tune=None):
        q, qd, qdd = q.contiguous(), qd.contiguous(), qdd.contiguous()
        kern = (tune or Tune()).kernel
        if kern in (L.WB_KERNEL_AUTO, L.WB_KERNEL_TREE, L.WB_KERNEL_TREE_NOCULL):
            o = robot.eval(q, qd, qdd, tune=tune, sphere=False, dmin=False)
            o.update({k: v for k, v in robot.self_collision(o["pose"], diff=True).items()
                      if k in ("sphere", "dmin", "worst", "diff")})
        else:
            o = robot.eval(q, qd, qdd, tune=tune)
            o["diff"] = None
        ctx.robot = robot
        ctx.tune = tune
        ctx.has_diff = o["diff"] is not None
        ctx.save_for_backward(q, qd, qdd, o["worst"],
                              o["diff"] if ctx.has_diff else o["worst"])
        ctx.mark_non_differentiable(o["worst"])
        return o["pose"], o["sphere"], o["dmin"], o["tau"], o["worst"]

    @staticmethod
    def backward(ctx, g_pose, g_sph, g_dmin, g_tau, _g_worst):
        q, qd, qdd, worst, diff = ctx.saved_tensors
        gq, gqd, gqdd = ctx.robot.eval_backward(q, qd, qdd, worst, _c(g_pose), _c(g_sph),
                                                _c(g_dmin), _c(g_tau), tune=ctx.tune,
                                                worst_diff=diff if ctx.has_diff else None)
        return None, gq, gqd, gqdd, None


def whole_body_eval(robot: Robot, q, qd, qdd, tune=None):
    """Differentiable evaluation: returns (link_pose, sphere, d_min, tau, worst)."""
    return WholeBodyEval.apply(robot, q, qd, qdd, tune)
