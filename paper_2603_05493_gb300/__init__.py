"""GB300-native whole-body evaluation (FK, sphere placement, self-collision
map-reduce, RNEA and their adjoints) for high-DoF robot motion generation.

The compute lives in libwbe.so (hand-written sm_103a CUDA kernels behind the
C ABI of include/wbe.h); `wbe` is a thin torch binding, imported on first use.
"""
import importlib

from .build import build  # noqa: F401

__all__ = ["build", "wbe"]


def __getattr__(name):
    if name == "wbe":
        return importlib.import_module(__name__ + ".wbe")
    raise AttributeError(name)
