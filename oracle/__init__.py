"""FP64 CPU oracle for batched edge validation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the package smoke check (``__graft_entry__.smoke``) and the
benchmark's CPU-baseline leg may import this package.  It wraps the plain C
implementation in ``vp_oracle.c`` (double precision, linear order, no sphere
hierarchy, no rake), which shares no code with the CUDA library.

What each function follows in arXiv 2309.14545:

* ``fk`` / ``link_frames`` -- Sec. "Vectorized Forward Kinematics": link poses
  composed joint by joint; only sphere positions are needed (Sec. "Vectorized
  Collision Checking", last paragraph).
* ``dist_*`` / ``clearance`` -- Sec. "Vectorized Collision Checking":
  sphere-based robot against sphere / capsule / cuboid primitives plus self
  pairs.
* ``edge_count`` / ``edge_states`` / ``validate_edges`` -- Sec. "Vectorized
  Motion Validation" (an edge is valid iff every state of its discretisation
  is valid) and Sec. "Bringing it Together" (linear interpolation in a
  Euclidean C-space).
* ``cost`` -- the penetration cost and its gradient, an addition beside the
  paper (no passage defines it).
* ``oracle.nn.nearest`` -- Sec. "Bringing it Together": l2 nearest neighbours
  in a Euclidean configuration space, brute force (NumPy, FP64).
* ``oracle.shortcut.shortcut`` -- Sec. "Bringing it Together": randomized
  shortcutting, batched over paths, on the FP64 edge check above.
* ``oracle.rrt.rrt_connect`` -- Sec. "Bringing it Together": RRT-Connect for
  one problem, on the FP64 edge check, with float32 nearest-node and
  steering arithmetic (the decisions the GPU takes in the same precision).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BAND = 1e-4  # clearance band (m) inside which a verdict is not pinned


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (IEEE double, no contraction)."""
    newer = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "vp_oracle.h")))
    if force or not newer:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Robot(C.Structure):
    _fields_ = [("n_joints", C.c_int32), ("parent", C.c_void_p), ("type", C.c_void_p),
                ("axis", C.c_void_p), ("origin", C.c_void_p), ("n_spheres", C.c_int32),
                ("sphere_link", C.c_void_p), ("sphere_centre", C.c_void_p),
                ("sphere_radius", C.c_void_p), ("n_pairs", C.c_int32), ("pairs", C.c_void_p)]


class _Env(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("spheres", C.c_void_p), ("n_capsules", C.c_int32),
                ("capsules", C.c_void_p), ("n_cuboids", C.c_int32), ("cuboids", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # VP_ORACLE_LIB: a prebuilt copy to load instead (the mutation
            # test points it at a copy with a planted mistake)
            lib = C.CDLL(os.environ.get("VP_ORACLE_LIB") or build())
            P, I64, I32, D, F = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_float
            sig = {
                "vpo_link_frames": (None, [P, P, P]),
                "vpo_fk_batch": (None, [P, P, I64, P]),
                "vpo_dist_sphere": (D, [P, P]),
                "vpo_dist_capsule": (D, [P, P]),
                "vpo_dist_cuboid": (D, [P, P]),
                "vpo_clearance_batch": (None, [P, P, P, I64, P]),
                "vpo_edge_count": (I32, [P, P, I32, F]),
                "vpo_edge_state": (None, [P, P, I32, I32, I32, P]),
                "vpo_edge_valid": (C.c_int, [P, P, P, P, I32]),
                "vpo_validate_edges": (I64, [P, P, P, P, P, F, I64, P]),
                "vpo_edge_classify": (C.c_int, [P, P, P, P, I32, D, P, P]),
                "vpo_classify_edges": (None, [P, P, P, P, P, F, I64, D, P, P]),
                "vpo_cost_batch": (None, [P, P, P, I64, D, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def _f64(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def _threads(n_threads):
    return max(1, int(n_threads if n_threads else os.cpu_count() or 1))


class Oracle:
    """The oracle bound to one robot and one environment (``vpgen`` arrays)."""

    def __init__(self, robot, env):
        self.lib = _load()
        D, S = robot.dof, robot.n_spheres
        self._keep = dict(
            parent=np.ascontiguousarray(robot.joint_parent, dtype=np.int32),
            type=np.ascontiguousarray(robot.joint_type, dtype=np.int32),
            axis=_f64(robot.joint_axis, (D, 3)),
            origin=_f64(robot.joint_origin, (D, 3, 4)),
            sphere_link=np.ascontiguousarray(robot.sphere_link, dtype=np.int32),
            sphere_centre=_f64(robot.sphere_centre, (S, 3)),
            sphere_radius=_f64(robot.sphere_radius, (S,)),
            pairs=np.ascontiguousarray(np.asarray(robot.self_pairs, dtype=np.int32).reshape(-1, 2)),
            spheres=_f64(env.spheres).reshape(-1, 4),
            capsules=_f64(env.capsules).reshape(-1, 7),
            cuboids=_f64(env.cuboids).reshape(-1, 15),
        )
        k = self._keep
        self.D, self.S = D, S
        self._robot = _Robot(D, _ptr(k["parent"]), _ptr(k["type"]), _ptr(k["axis"]), _ptr(k["origin"]),
                             S, _ptr(k["sphere_link"]), _ptr(k["sphere_centre"]), _ptr(k["sphere_radius"]),
                             k["pairs"].shape[0], _ptr(k["pairs"]))
        self._env = _Env(k["spheres"].shape[0], _ptr(k["spheres"]), k["capsules"].shape[0],
                         _ptr(k["capsules"]), k["cuboids"].shape[0], _ptr(k["cuboids"]))
        self._rp = C.cast(C.pointer(self._robot), C.c_void_p)
        self._ep = C.cast(C.pointer(self._env), C.c_void_p)

    # -- kinematics --------------------------------------------------------
    def link_frames(self, q):
        q = _f64(q, (self.D,))
        out = np.zeros((self.D + 1, 3, 4))
        self.lib.vpo_link_frames(self._rp, _ptr(q), _ptr(out))
        return out

    def fk(self, q):
        """World sphere centres [N, S, 3] for configurations q [N, D]."""
        q = _f64(q).reshape(-1, self.D)
        out = np.zeros((q.shape[0], self.S, 3))
        if q.shape[0]:
            self.lib.vpo_fk_batch(self._rp, _ptr(q), q.shape[0], _ptr(out))
        return out

    # -- distances ---------------------------------------------------------
    def dist_sphere(self, x, sphere):
        return self.lib.vpo_dist_sphere(_ptr(_f64(x, (3,))), _ptr(_f64(sphere, (4,))))

    def dist_capsule(self, x, capsule):
        return self.lib.vpo_dist_capsule(_ptr(_f64(x, (3,))), _ptr(_f64(capsule, (7,))))

    def dist_cuboid(self, x, cuboid):
        return self.lib.vpo_dist_cuboid(_ptr(_f64(x, (3,))), _ptr(_f64(cuboid, (15,))))

    # -- states ------------------------------------------------------------
    def clearance(self, q, n_threads=None):
        """Clearance K(q) [N] (state valid iff K >= 0)."""
        q = _f64(q).reshape(-1, self.D)
        out = np.zeros(q.shape[0])
        self._parallel(q.shape[0], n_threads, lambda a, b: self.lib.vpo_clearance_batch(
            self._rp, self._ep, _ptr(q[a:b]), b - a, _ptr(out[a:b])))
        return out

    # -- edges -------------------------------------------------------------
    def edge_count(self, q0, q1, res):
        q0 = np.ascontiguousarray(q0, dtype=np.float32).reshape(-1, self.D)
        q1 = np.ascontiguousarray(q1, dtype=np.float32).reshape(-1, self.D)
        return np.array([self.lib.vpo_edge_count(_ptr(q0[i]), _ptr(q1[i]), self.D, C.c_float(res))
                         for i in range(q0.shape[0])], dtype=np.int32)

    def edge_states(self, q0, q1, k):
        """All k states of one edge [k, D], in double."""
        q0 = np.ascontiguousarray(q0, dtype=np.float32).reshape(self.D)
        q1 = np.ascontiguousarray(q1, dtype=np.float32).reshape(self.D)
        out = np.zeros((k, self.D))
        for i in range(k):
            self.lib.vpo_edge_state(_ptr(q0), _ptr(q1), self.D, k, i, _ptr(out[i]))
        return out

    def validate_edges(self, q0, q1, counts=None, res=1.0 / 32.0, n_threads=None):
        """Edge verdicts uint8 [E] (1 = every state valid), linear order."""
        q0 = np.ascontiguousarray(q0, dtype=np.float32).reshape(-1, self.D)
        q1 = np.ascontiguousarray(q1, dtype=np.float32).reshape(-1, self.D)
        counts = None if counts is None else np.ascontiguousarray(counts, dtype=np.int32)
        E = q0.shape[0]
        out = np.zeros(E, dtype=np.uint8)
        self._parallel(E, n_threads, lambda a, b: self.lib.vpo_validate_edges(
            self._rp, self._ep, _ptr(q0[a:b]), _ptr(q1[a:b]),
            None if counts is None else _ptr(counts[a:b]), C.c_float(res), b - a, _ptr(out[a:b])))
        return out

    def classify_edges(self, q0, q1, counts=None, res=1.0 / 32.0, band=BAND, n_threads=None):
        """(class int8 [E], band-state count int32 [E]): 0 pinned free,
        1 pinned collide, 2 band."""
        q0 = np.ascontiguousarray(q0, dtype=np.float32).reshape(-1, self.D)
        q1 = np.ascontiguousarray(q1, dtype=np.float32).reshape(-1, self.D)
        counts = None if counts is None else np.ascontiguousarray(counts, dtype=np.int32)
        E = q0.shape[0]
        cls = np.zeros(E, dtype=np.int8)
        nb = np.zeros(E, dtype=np.int32)
        self._parallel(E, n_threads, lambda a, b: self.lib.vpo_classify_edges(
            self._rp, self._ep, _ptr(q0[a:b]), _ptr(q1[a:b]),
            None if counts is None else _ptr(counts[a:b]), C.c_float(res), b - a, C.c_double(band),
            _ptr(cls[a:b]), _ptr(nb[a:b])))
        return cls, nb

    # -- cost --------------------------------------------------------------
    def cost(self, q, margin, grad=True, n_threads=None):
        """Penetration cost [N] and, if ``grad``, dc/dq [N, D]."""
        q = _f64(q).reshape(-1, self.D)
        N = q.shape[0]
        c = np.zeros(N)
        g = np.zeros((N, self.D)) if grad else None
        self._parallel(N, n_threads, lambda a, b: self.lib.vpo_cost_batch(
            self._rp, self._ep, _ptr(q[a:b]), b - a, C.c_double(margin), _ptr(c[a:b]),
            None if g is None else _ptr(g[a:b])))
        return (c, g) if grad else c

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _parallel(n, n_threads, fn):
        """Run fn(a, b) over [0, n) in chunks on a thread pool (ctypes releases the GIL)."""
        if n == 0:
            return
        t = min(_threads(n_threads), n)
        if t == 1:
            fn(0, n)
            return
        chunk = max(1, (n + 4 * t - 1) // (4 * t))
        bounds = [(a, min(n, a + chunk)) for a in range(0, n, chunk)]
        with ThreadPoolExecutor(max_workers=t) as ex:
            list(ex.map(lambda ab: fn(*ab), bounds))
