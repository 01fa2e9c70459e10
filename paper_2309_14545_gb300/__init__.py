"""GPU-native batched motion (edge) validation for sampling-based planning.

The hot path of arXiv 2309.14545 ("Motions in Microseconds via Vectorized
Sampling-Based Planning"): raked edge interpolation, FK to collision
spheres, hierarchical sphere checks against environment primitives and self
pairs, and early exit -- as hand-written CUDA kernels for sm_103a behind the
C ABI in include/vp.h.  ``vp`` is the thin ctypes binding (same names as the
C calls); ``Validator`` owns a context; ``CollisionCost`` wraps the
penetration cost and its FK adjoint as a torch.autograd.Function.
"""
from .api import CollisionCost, Validator  # noqa: F401
