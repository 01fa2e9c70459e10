"""Thin ctypes binding over libvp's C ABI (include/vp.h), same names.

Argument marshalling only: every step of edge validation runs in the CUDA
kernels of libvp.so.  PyTorch supplies device memory and streams.  If the
library has not been built, importing this module raises (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvp.so")

VP_OK, VP_ERR_ARG, VP_ERR_CUDA, VP_ERR_CAPACITY, VP_ERR_NOT_LOADED, VP_ERR_TIMEOUT, VP_ERR_DEVICE = range(7)
STATUS_NAMES = ["VP_OK", "VP_ERR_ARG", "VP_ERR_CUDA", "VP_ERR_CAPACITY", "VP_ERR_NOT_LOADED",
                "VP_ERR_TIMEOUT", "VP_ERR_DEVICE"]
VP_MODE_PLAIN, VP_MODE_BATCHED, VP_MODE_PER_EDGE = 0, 1, 2
VP_DEVERR_COUNT, VP_DEVERR_LENGTH, VP_DEVERR_TIMEOUT = 0x1, 0x2, 0x4
VP_ORDER_PRIMS_FIRST, VP_ORDER_INTERLEAVE, VP_ORDER_FREQUENT = 0x1, 0x2, 0x4
VP_ORDER_FREQUENT_TWO_PASS = 5
VP_MAX_JOINTS, VP_MAX_SPHERES, VP_MAX_PAIRS = 16, 256, 1024
VP_MAX_ENV_BYTES = 160 * 1024
VP_NOALLOC_MAX_ENV_BYTES = 64 * 1024
VP_MAX_STEPS = 16777216
(VP_WORK_STATES, VP_WORK_LINK_CENTRES, VP_WORK_COARSE_SPHERE, VP_WORK_COARSE_CAPSULE, VP_WORK_COARSE_CUBOID,
 VP_WORK_FINE_SPHERE, VP_WORK_FINE_CAPSULE, VP_WORK_FINE_CUBOID, VP_WORK_PAIR_COARSE, VP_WORK_PAIR_FINE,
 VP_WORK_EDGES_DONE, VP_WORK_LANE_STATES, VP_WORK_LANE_COARSE, VP_WORK_LANE_FINE,
 VP_WORK_LANE_PAIR_FINE, VP_WORK_BOX_TESTS, VP_WORK_FINE_OWN, VP_WORK_PAIR_FINE_OWN) = range(18)
VP_WORK_N = 32

#: Every symbol include/vp.h declares.
EXPORTS = ("vp_create", "vp_destroy", "vp_last_error", "vp_load_robot", "vp_load_env", "vp_fk_spheres",
           "vp_validate_states", "vp_edge_counts", "vp_validate_edges", "vp_validate_edges_work",
           "vp_collision_cost", "vp_autotune", "vp_sync_status", "vp_validate_edges_noalloc",
           "vp_kernel_time", "vp_set_watchdog", "vp_tiling", "vp_set_tiling", "vp_set_screen_rounds",
           "vp_screen_rounds", "vp_set_check_order", "vp_check_order", "vp_measure_fp32_peak", "vp_nearest",
           "vp_shortcut_paths", "vp_rrt_connect", "vp_fk_codegen", "vp_link_bounds", "vp_validate_edges_host")


class VPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")
        self.status = status


class vp_robot_desc(C.Structure):
    _fields_ = [("n_joints", C.c_int32), ("joint_parent", C.c_void_p), ("joint_type", C.c_void_p),
                ("joint_axis", C.c_void_p), ("joint_origin", C.c_void_p), ("n_spheres", C.c_int32),
                ("sphere_link", C.c_void_p), ("sphere_centre", C.c_void_p), ("sphere_radius", C.c_void_p),
                ("link_spheres", C.c_void_p), ("n_pairs", C.c_int32), ("self_pairs", C.c_void_p)]


class vp_env_desc(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("spheres", C.c_void_p), ("n_capsules", C.c_int32),
                ("capsules", C.c_void_p), ("n_cuboids", C.c_int32), ("cuboids", C.c_void_p)]


def _load_lib():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2309_14545_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P, I64, I32, F, U = C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_int
    sig = {
        "vp_create": (U, [C.POINTER(C.c_void_p), U]),
        "vp_destroy": (U, [P]),
        "vp_last_error": (C.c_char_p, [P]),
        "vp_load_robot": (U, [P, P]),
        "vp_load_env": (U, [P, P]),
        "vp_fk_spheres": (U, [P, P, I64, P, P]),
        "vp_validate_states": (U, [P, P, I64, P, P]),
        "vp_edge_counts": (U, [P, P, P, F, I64, P, P]),
        "vp_validate_edges": (U, [P, P, P, P, F, I64, P, U, P]),
        "vp_validate_edges_work": (U, [P, P, P, P, F, I64, P, U, P, P]),
        "vp_collision_cost": (U, [P, P, I64, F, P, P, P]),
        "vp_autotune": (U, [P, P, P, P, F, I64, P]),
        "vp_sync_status": (U, [P, P, C.POINTER(C.c_uint32)]),
        "vp_validate_edges_noalloc": (U, [P, P, P, P, P, F, I64, P, P, C.c_char_p, I32]),
        "vp_kernel_time": (U, [P, U, C.POINTER(C.c_float)]),
        "vp_set_watchdog": (U, [P, C.c_double]),
        "vp_tiling": (U, [P, C.POINTER(C.c_int32), C.c_int, C.POINTER(C.c_int)]),
        "vp_set_tiling": (U, [P, C.POINTER(C.c_int32), C.c_int]),
        "vp_set_screen_rounds": (U, [P, C.c_int]),
        "vp_screen_rounds": (U, [P, C.POINTER(C.c_int)]),
        "vp_set_check_order": (U, [P, C.c_int]),
        "vp_check_order": (U, [P, C.POINTER(C.c_int)]),
        "vp_measure_fp32_peak": (U, [C.c_int, C.c_double, C.POINTER(C.c_double)]),
        "vp_nearest": (U, [P, P, I64, P, I64, C.c_int, P, P, P]),
        "vp_shortcut_paths": (U, [P, P, P, I64, C.c_int32, P, C.c_int32, F, P]),
        "vp_rrt_connect": (U, [P, P, P, I64, P, C.c_int32, F, F, C.c_int32, P, P, P, P, P, P]),
        "vp_fk_codegen": (U, [P, C.c_int, C.POINTER(C.c_double)]),
        "vp_link_bounds": (U, [P, C.c_int, P, P, P]),
        "vp_validate_edges_host": (U, [P, P, P, P, F, I64, P, C.c_int, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load_lib()


def _check(ctx, status):
    if status != VP_OK:
        msg = lib.vp_last_error(ctx)
        raise VPError(status, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev(t, dtype, name, shape=None):
    """Device pointer of a contiguous CUDA tensor of the given dtype (None -> NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr() if t.numel() else None


def _host(t, dtype, name, shape=None):
    """Host pointer of a contiguous CPU tensor of the given dtype (None -> NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a CPU tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr() if t.numel() else None


# ---------------------------------------------------------------------------
# the C calls, same names

def vp_create(device: int = 0):
    h = C.c_void_p()
    st = lib.vp_create(C.byref(h), int(device))
    if st != VP_OK:
        raise VPError(st, f"vp_create(device={device}) failed")
    return h


def vp_destroy(ctx):
    lib.vp_destroy(ctx)


def vp_last_error(ctx) -> str:
    m = lib.vp_last_error(ctx)
    return m.decode() if m else ""


def _arr(x, dtype, shape):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype).reshape(shape))


def vp_load_robot(ctx, robot):
    """robot: an object with the vp_robot_desc fields as arrays (e.g. vpgen.Robot)."""
    D = int(np.asarray(robot.joint_type).shape[0])
    S = int(np.asarray(robot.sphere_radius).shape[0])
    pairs = _arr(robot.self_pairs, np.int32, (-1, 2))
    keep = [
        _arr(robot.joint_parent, np.int32, (D,)), _arr(robot.joint_type, np.int32, (D,)),
        _arr(robot.joint_axis, np.float64, (D, 3)), _arr(robot.joint_origin, np.float64, (D, 3, 4)),
        _arr(robot.sphere_link, np.int32, (S,)), _arr(robot.sphere_centre, np.float64, (S, 3)),
        _arr(robot.sphere_radius, np.float64, (S,)),
        None if getattr(robot, "link_spheres", None) is None else _arr(robot.link_spheres, np.float64, (D + 1, 4)),
        pairs,
    ]
    ptr = [None if a is None or a.size == 0 else a.ctypes.data for a in keep]
    desc = vp_robot_desc(D, ptr[0], ptr[1], ptr[2], ptr[3], S, ptr[4], ptr[5], ptr[6], ptr[7],
                         pairs.shape[0], ptr[8])
    _check(ctx, lib.vp_load_robot(ctx, C.byref(desc)))


def vp_load_env(ctx, env):
    """env: an object with spheres [n,4], capsules [n,7], cuboids [n,15] (e.g. vpgen.Env)."""
    s = _arr(env.spheres, np.float64, (-1, 4))
    c = _arr(env.capsules, np.float64, (-1, 7))
    b = _arr(env.cuboids, np.float64, (-1, 15))
    p = [a.ctypes.data if a.size else None for a in (s, c, b)]
    desc = vp_env_desc(s.shape[0], p[0], c.shape[0], p[1], b.shape[0], p[2])
    _check(ctx, lib.vp_load_env(ctx, C.byref(desc)))


def vp_fk_spheres(ctx, q, centres, stream=None):
    n = q.shape[0]
    _check(ctx, lib.vp_fk_spheres(ctx, _dev(q, torch.float32, "q"), n,
                                  _dev(centres, torch.float32, "centres"), _stream(stream)))


def vp_validate_states(ctx, q, valid, stream=None):
    n = q.shape[0]
    _check(ctx, lib.vp_validate_states(ctx, _dev(q, torch.float32, "q"), n,
                                       _dev(valid, torch.uint8, "valid", (n,)), _stream(stream)))


def vp_edge_counts(ctx, q0, q1, resolution, counts, stream=None):
    E = q0.shape[0]
    _check(ctx, lib.vp_edge_counts(ctx, _dev(q0, torch.float32, "q0"), _dev(q1, torch.float32, "q1", q0.shape),
                                   C.c_float(resolution), E, _dev(counts, torch.int32, "counts", (E,)),
                                   _stream(stream)))


def vp_validate_edges(ctx, q0, q1, counts, resolution, valid, mode=VP_MODE_PLAIN, stream=None):
    E = q0.shape[0]
    _check(ctx, lib.vp_validate_edges(ctx, _dev(q0, torch.float32, "q0"),
                                      _dev(q1, torch.float32, "q1", q0.shape),
                                      _dev(counts, torch.int32, "counts", (E,)), C.c_float(resolution), E,
                                      _dev(valid, torch.uint8, "valid", (E,)), int(mode), _stream(stream)))


def vp_validate_edges_host(ctx, q0, q1, counts, resolution, valid, mode=VP_MODE_PLAIN, stream=None):
    """q0, q1, counts, valid: CPU tensors (page-locked for overlapped copies);
    the verdicts are in valid once `stream` has completed."""
    E = q0.shape[0]
    _check(ctx, lib.vp_validate_edges_host(ctx, _host(q0, torch.float32, "q0"),
                                           _host(q1, torch.float32, "q1", q0.shape),
                                           _host(counts, torch.int32, "counts", (E,)), C.c_float(resolution), E,
                                           _host(valid, torch.uint8, "valid", (E,)), int(mode), _stream(stream)))


def vp_validate_edges_work(ctx, q0, q1, counts, resolution, valid, mode, work, stream=None):
    E = q0.shape[0]
    _check(ctx, lib.vp_validate_edges_work(ctx, _dev(q0, torch.float32, "q0"),
                                           _dev(q1, torch.float32, "q1", q0.shape),
                                           _dev(counts, torch.int32, "counts", (E,)), C.c_float(resolution), E,
                                           _dev(valid, torch.uint8, "valid", (E,)), int(mode),
                                           _dev(work, torch.int64, "work", (VP_WORK_N,)), _stream(stream)))


def vp_collision_cost(ctx, q, margin, cost, grad=None, stream=None):
    n = q.shape[0]
    _check(ctx, lib.vp_collision_cost(ctx, _dev(q, torch.float32, "q"), n, C.c_float(margin),
                                      _dev(cost, torch.float32, "cost", (n,)),
                                      _dev(grad, torch.float32, "grad", q.shape), _stream(stream)))


def vp_autotune(ctx, q0, q1, counts, resolution, stream=None):
    E = q0.shape[0]
    _check(ctx, lib.vp_autotune(ctx, _dev(q0, torch.float32, "q0"), _dev(q1, torch.float32, "q1", q0.shape),
                                _dev(counts, torch.int32, "counts", (E,)), C.c_float(resolution), E,
                                _stream(stream)))


def vp_kernel_time(ctx, enable=True):
    """Enable/disable kernel timing; returns the last timed kernel's ms (-1 if none)."""
    ms = C.c_float(-1.0)
    _check(ctx, lib.vp_kernel_time(ctx, int(bool(enable)), C.byref(ms)))
    return ms.value


def vp_set_watchdog(ctx, seconds):
    _check(ctx, lib.vp_set_watchdog(ctx, C.c_double(seconds)))


def vp_tiling(ctx):
    """Lanes per edge of each edge-length bucket of the batched mode."""
    arr = (C.c_int32 * 16)()
    nb = C.c_int(0)
    _check(ctx, lib.vp_tiling(ctx, arr, 16, C.byref(nb)))
    return [int(arr[b]) for b in range(min(nb.value, 16))]


def vp_set_tiling(ctx, lanes):
    """Set lanes per edge for the first len(lanes) buckets (each 4, 8, 16 or 32)."""
    lanes = [int(x) for x in lanes]
    arr = (C.c_int32 * max(1, len(lanes)))(*lanes)
    _check(ctx, lib.vp_set_tiling(ctx, arr, len(lanes)))


def vp_set_screen_rounds(ctx, rounds):
    _check(ctx, lib.vp_set_screen_rounds(ctx, int(rounds)))


def vp_screen_rounds(ctx):
    r = C.c_int(0)
    _check(ctx, lib.vp_screen_rounds(ctx, C.byref(r)))
    return r.value


def vp_set_check_order(ctx, order):
    _check(ctx, lib.vp_set_check_order(ctx, int(order)))


def vp_check_order(ctx):
    r = C.c_int(0)
    _check(ctx, lib.vp_check_order(ctx, C.byref(r)))
    return r.value


def vp_link_bounds(ctx, n_links, n_spheres):
    """The packed link spheres, half spheres and each sphere's half (numpy)."""
    link = np.zeros((n_links, 4), dtype=np.float32)
    half = np.zeros((n_links, 2, 4), dtype=np.float32)
    which = np.zeros(n_spheres, dtype=np.int32)
    _check(ctx, lib.vp_link_bounds(ctx, int(n_links), link.ctypes.data, half.ctypes.data, which.ctypes.data))
    return link, half, which


def vp_nearest(ctx, points, queries, index, dist2=None, stream=None):
    """l2 nearest neighbour of each query among the points (device tensors)."""
    if points.dim() != 2 or queries.dim() != 2 or points.shape[1] != queries.shape[1]:
        raise ValueError("points [M, D] and queries [N, D]")
    M, D = points.shape
    N = queries.shape[0]
    _check(ctx, lib.vp_nearest(ctx, _dev(points, torch.float32, "points", (M, D)), M,
                               _dev(queries, torch.float32, "queries", (N, D)), N, D,
                               _dev(index, torch.int64, "index", (N,)),
                               None if dist2 is None else _dev(dist2, torch.float32, "dist2", (N,)),
                               _stream(stream)))


def vp_shortcut_paths(ctx, paths, lengths, draws, resolution=1.0 / 32.0, stream=None):
    """Randomized shortcutting in place: paths [P, W, D], lengths [P] int32,
    draws [T, P, 2] float32 (device tensors)."""
    if paths.dim() != 3 or draws.dim() != 3:
        raise ValueError("paths [P, W, D] and draws [T, P, 2]")
    P_, W, D = paths.shape
    T = draws.shape[0]
    _check(ctx, lib.vp_shortcut_paths(ctx, _dev(paths, torch.float32, "paths", (P_, W, D)),
                                      _dev(lengths, torch.int32, "lengths", (P_,)), P_, W,
                                      _dev(draws, torch.float32, "draws", (T, P_, 2)), T, C.c_float(resolution),
                                      _stream(stream)))


def vp_rrt_connect(ctx, start, goal, samples, range_, resolution, cap, status, iters, path, path_len, tree_sizes,
                   stream=None):
    """Batched RRT-Connect on device tensors (see include/vp.h)."""
    B, D = start.shape
    T = samples.shape[1]
    _check(ctx, lib.vp_rrt_connect(ctx, _dev(start, torch.float32, "start", (B, D)),
                                   _dev(goal, torch.float32, "goal", (B, D)), B,
                                   _dev(samples, torch.float32, "samples", (B, T, D)), T, C.c_float(range_),
                                   C.c_float(resolution), int(cap), _dev(status, torch.int32, "status", (B,)),
                                   _dev(iters, torch.int32, "iters", (B,)),
                                   _dev(path, torch.float32, "path", (B, 2 * cap, D)),
                                   _dev(path_len, torch.int32, "path_len", (B,)),
                                   _dev(tree_sizes, torch.int32, "tree_sizes", (B, 2)), _stream(stream)))


def vp_fk_codegen(ctx, enable=True):
    """Choose vp_fk_spheres' kernel: 1 (True) the per-robot generated one,
    0 (False) the table-driven one, -1 automatic; returns the generation and
    compile time in ms."""
    ms = C.c_double(0.0)
    _check(ctx, lib.vp_fk_codegen(ctx, int(enable), C.byref(ms)))
    return ms.value


def vp_measure_fp32_peak(device=0, seconds=1.0):
    """Measured FP32 FMA throughput of `device` (TFLOP/s)."""
    t = C.c_double(0.0)
    status = lib.vp_measure_fp32_peak(int(device), C.c_double(seconds), C.byref(t))
    if status != VP_OK:
        raise VPError(status, "vp_measure_fp32_peak failed")
    return t.value


def vp_sync_status(ctx, stream=None):
    """Returns (status, bits) without raising."""
    bits = C.c_uint32(0)
    st = lib.vp_sync_status(ctx, _stream(stream), C.byref(bits))
    return st, bits.value


def vp_validate_edges_noalloc(robot, env, q0, q1, counts, resolution, valid, stream=None):
    """Edge validation without a context and without device allocation (see
    include/vp.h): the packed environment and the status word live in a
    static device array of the library.  Synchronous on `stream`."""
    E = q0.shape[0]
    D = int(np.asarray(robot.joint_type).shape[0])
    S = int(np.asarray(robot.sphere_radius).shape[0])
    pairs = _arr(robot.self_pairs, np.int32, (-1, 2))
    keep = [
        _arr(robot.joint_parent, np.int32, (D,)), _arr(robot.joint_type, np.int32, (D,)),
        _arr(robot.joint_axis, np.float64, (D, 3)), _arr(robot.joint_origin, np.float64, (D, 3, 4)),
        _arr(robot.sphere_link, np.int32, (S,)), _arr(robot.sphere_centre, np.float64, (S, 3)),
        _arr(robot.sphere_radius, np.float64, (S,)),
        None if getattr(robot, "link_spheres", None) is None else _arr(robot.link_spheres, np.float64, (D + 1, 4)),
        pairs,
    ]
    ptr = [None if a is None or a.size == 0 else a.ctypes.data for a in keep]
    rdesc = vp_robot_desc(D, ptr[0], ptr[1], ptr[2], ptr[3], S, ptr[4], ptr[5], ptr[6], ptr[7],
                          pairs.shape[0], ptr[8])
    s = _arr(env.spheres, np.float64, (-1, 4))
    c = _arr(env.capsules, np.float64, (-1, 7))
    b = _arr(env.cuboids, np.float64, (-1, 15))
    p = [a.ctypes.data if a.size else None for a in (s, c, b)]
    edesc = vp_env_desc(s.shape[0], p[0], c.shape[0], p[1], b.shape[0], p[2])
    buf = C.create_string_buffer(512)
    st = lib.vp_validate_edges_noalloc(C.byref(rdesc), C.byref(edesc), _dev(q0, torch.float32, "q0"),
                                       _dev(q1, torch.float32, "q1", q0.shape),
                                       _dev(counts, torch.int32, "counts", (E,)), C.c_float(resolution), E,
                                       _dev(valid, torch.uint8, "valid", (E,)), _stream(stream), buf, 512)
    if st != VP_OK:
        raise VPError(st, buf.value.decode())
