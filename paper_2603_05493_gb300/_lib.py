"""ctypes declarations of the C ABI in include/wbe.h (argument marshalling
only).  Loading fails loudly if libwbe.so has not been built: there is no
fallback implementation."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwbe.so")

WB_OK = 0
WB_EINVAL = -1
WB_ETOPO = -2
WB_ERANGE = -3
WB_ETOOBIG = -4
WB_EDEVICE = -5
WB_ECUDA = -6
ERRNAMES = {0: "WB_OK", -1: "WB_EINVAL", -2: "WB_ETOPO", -3: "WB_ERANGE", -4: "WB_ETOOBIG",
            -5: "WB_EDEVICE", -6: "WB_ECUDA"}

WB_KERNEL_AUTO = 0
WB_KERNEL_PLAIN = 1
WB_KERNEL_FUSED = 2
WB_KERNEL_TREE = 3
WB_KERNEL_TREE_NOCULL = 4

p = C.c_void_p


class wb_tree(C.Structure):
    _fields_ = [("n_links", C.c_int32), ("parent", p), ("joint_type", p), ("axis", p),
                ("T_fixed", p), ("joint_index", p), ("mimic_mult", p), ("mimic_offset", p),
                ("gravity", p)]


class wb_spheres(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("link", p), ("center", p), ("radius", p)]


class wb_pairs(C.Structure):
    _fields_ = [("n_pairs", C.c_int32), ("pairs", p), ("mask", p)]


class wb_inertial(C.Structure):
    _fields_ = [("mass", p), ("com", p), ("inertia", p), ("n_points", C.c_int32),
                ("point_link", p), ("point_mass", p), ("point_pos", p)]


class wb_tune(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("lanes_per_config", C.c_int32),
                ("configs_per_block", C.c_int32), ("blocks_per_sm", C.c_int32)]


class wb_cost_weights(C.Structure):
    _fields_ = [("collision", C.c_float), ("smooth", C.c_float), ("length", C.c_float),
                ("energy", C.c_float), ("dt", C.c_float)]


class wb_spline(C.Structure):
    _fields_ = [("U", C.c_void_p), ("n_traj", C.c_int64), ("K", C.c_int32), ("T", C.c_int32),
                ("dt", C.c_float)]


class wb_problem(C.Structure):
    _fields_ = [("robot", C.c_int32), ("horizon", C.c_int32)]


class wb_batch_sizes(C.Structure):
    _fields_ = [("joint_elems", C.c_int64), ("pose_elems", C.c_int64),
                ("sphere_elems", C.c_int64), ("configs", C.c_int64),
                ("n_problems", C.c_int32), ("n_robots", C.c_int32)]


class wb_batch_tune(C.Structure):
    _fields_ = [("fwd_threads", C.c_int32), ("bwd_threads", C.c_int32),
                ("pair_warps", C.c_int32)]


class wb_robot_info(C.Structure):
    _fields_ = [("n_links", C.c_int32), ("dof", C.c_int32), ("n_spheres", C.c_int32),
                ("n_pairs", C.c_int32), ("n_levels", C.c_int32), ("max_level_width", C.c_int32),
                ("n_pair_blocks", C.c_int32), ("device", C.c_int32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "wb_version": (C.c_int, []),
    "wb_last_error": (C.c_char_p, []),
    "wb_load_robot": (C.c_int, [C.POINTER(wb_tree), C.POINTER(wb_spheres), C.POINTER(wb_pairs),
                                C.POINTER(wb_inertial), C.c_int, C.POINTER(p)]),
    "wb_set_inertials": (C.c_int, [p, C.POINTER(wb_inertial), p]),
    "wb_robot_info_get": (C.c_int, [p, C.POINTER(wb_robot_info)]),
    "wb_plan_info": (C.c_int, [C.POINTER(wb_tree), C.POINTER(wb_spheres), C.POINTER(wb_pairs),
                               C.POINTER(wb_inertial), C.POINTER(wb_robot_info),
                               C.POINTER(C.c_int32)]),
    "wb_eval": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, p, p, p, C.POINTER(wb_tune), p]),
    "wb_self_collision": (C.c_int, [p, C.c_int64, p, p, p, p, p, p]),
    "wb_eval_backward": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, p, p, p, p, p,
                                   C.POINTER(wb_tune), p]),
    "wb_free_robot": (None, [p]),
    "wb_autotune": (C.c_int, [p, C.c_int64, C.POINTER(wb_tune), C.POINTER(wb_tune),
                              C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "wb_batch_create": (C.c_int, [C.POINTER(p), C.c_int32, C.POINTER(wb_problem), C.c_int32,
                                  C.POINTER(p)]),
    "wb_batch_sizes_get": (C.c_int, [p, C.POINTER(wb_batch_sizes)]),
    "wb_batch_offsets": (C.c_int, [p, p, p, p, p]),
    "wb_batch_eval": (C.c_int, [p, p, p, p, p, p, p, p, p, p]),
    "wb_batch_eval_backward": (C.c_int, [p, p, p, p, p, p, p, p, p, p, p, p, p]),
    "wb_free_batch": (None, [p]),
    "wb_batch_set_tune": (C.c_int, [p, C.POINTER(wb_batch_tune), p, p]),
    "wb_batch_get_tune": (C.c_int, [p, C.POINTER(wb_batch_tune), p, p]),
    "wb_batch_autotune": (C.c_int, [p, C.POINTER(wb_batch_tune), p, p, C.POINTER(C.c_float),
                                    C.POINTER(C.c_float)]),
    "wb_batch_eval_noalloc": (C.c_int, [p, C.c_int32, p, C.c_int32, p, p, p, p, p, p, p, p, p]),
    "wb_bspline_eval": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_float, p, p, p,
                                  p, p]),
    "wb_bspline_backward": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_float, p,
                                      p, p, p, p]),
    "wb_trajopt_cost": (C.c_int, [C.c_int64, C.c_int32, p, p, p, p, C.c_float, p, p, p, p]),
    "wb_bspline_backward_ext": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                          p, p, p, p, p, p, p]),
    "wb_eval_spline": (C.c_int, [p, C.POINTER(wb_spline), p, p, p, p, p, C.POINTER(wb_tune),
                                 p]),
    "wb_eval_backward_spline_cost": (C.c_int, [p, C.POINTER(wb_spline), p, p, p, p, p, p, p,
                                               C.POINTER(wb_cost_weights), p, p, p, p,
                                               C.POINTER(wb_tune), p]),
    "wb_autotune_spline": (C.c_int, [p, C.c_int64, C.c_int32, C.c_int32, C.c_float,
                                     C.POINTER(wb_cost_weights), C.POINTER(wb_tune),
                                     C.POINTER(wb_tune), C.POINTER(C.c_float),
                                     C.POINTER(C.c_float)]),
    "wb_eval_backward_cost": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, p, p, p, p,
                                        C.POINTER(wb_cost_weights), p, p, p, p,
                                        C.POINTER(wb_tune), p]),
    "wb_eval_backward_cost_dir": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, p, p, p, p, p,
                                            C.POINTER(wb_cost_weights), p, p, p, p,
                                            C.POINTER(wb_tune), p]),
    "wb_eval_backward_spline_cost_dir": (C.c_int, [p, C.POINTER(wb_spline), p, p, p, p, p, p,
                                                   p, p, C.POINTER(wb_cost_weights), p, p, p,
                                                   p, C.POINTER(wb_tune), p]),
    "wb_bspline_eval_bc": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_float, p, p,
                                     C.c_int32, p, p, p, p]),
    "wb_bspline_backward_bc": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                         C.c_int32, C.c_int32, p, p, p, p, p, p, p, p]),
    "wb_trajopt_cost_ext": (C.c_int, [C.c_int64, C.c_int32, p, p, p, p, p, p,
                                      C.POINTER(wb_cost_weights), p, p, p, p, p, p]),
    "wb_self_collision_hinge": (C.c_int, [p, C.c_int64, p, C.c_float, C.c_float, p, p, p]),
    "wb_kinematics": (C.c_int, [p, C.c_int64, p, C.c_int32, p, p, p, p, p]),
    "wb_self_collision_tuned": (C.c_int, [p, C.c_int64, p, p, p, p, p, C.POINTER(wb_tune), p]),
    "wb_self_collision_dir": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, C.POINTER(wb_tune), p]),
    "wb_eval_backward_dir": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, p, p, p, p, p, p, p, p,
                                       C.POINTER(wb_tune), p]),
    "wb_eval_ext": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, p, p, p, p, C.POINTER(wb_tune), p]),
    "wb_eval_backward_ext": (C.c_int, [p, C.c_int64, p, p, p, p, p, p, p, p, p, p, p, p, p,
                                       C.POINTER(wb_tune), p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libwbe.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(
                "libwbe.so not found at %s: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')" % path)
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class WbError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed: %s (%s)" % (where, msg, ERRNAMES.get(code, code)))
        self.code = code


def check(code: int, where: str):
    if code != WB_OK:
        raise WbError(code, where, load().wb_last_error().decode(errors="replace"))
