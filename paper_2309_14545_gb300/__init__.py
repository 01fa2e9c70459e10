"""GPU-native batched motion (edge) validation for sampling-based planning.

The hot path of arXiv 2309.14545 ("Motions in Microseconds via Vectorized
Sampling-Based Planning"): raked edge interpolation, FK to collision
spheres, hierarchical sphere checks against environment primitives and self
pairs, and early exit -- as hand-written CUDA kernels for sm_103a behind the
C ABI in include/vp.h.  ``vp`` is the thin ctypes binding (same names as the
C calls); ``Validator`` owns a context; ``CollisionCost`` wraps the
penetration cost and its FK adjoint as a torch.autograd.Function.

``build`` compiles libvp.so; everything else loads it on first use and
raises if it is missing (there is no CPU fallback).
"""

__all__ = ["Validator", "CollisionCost", "vp", "build"]


def __getattr__(name):
    import importlib
    if name in ("Validator", "CollisionCost"):
        return getattr(importlib.import_module(".api", __name__), name)
    if name in ("vp", "build", "api"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
