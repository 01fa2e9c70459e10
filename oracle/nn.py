"""FP64 nearest neighbours -- TEST INFRASTRUCTURE ONLY (see the package
header: only tests/, the smoke check and the benchmark's CPU-baseline legs
use it).

Sec. III-E ("Bringing it Together"): the configuration space is Euclidean,
and the planners' nearest-neighbour structure measures the l2 distance, the
sum of squared coordinate differences.  The oracle is that definition, brute
force: every query against every point.
"""
from __future__ import annotations

import numpy as np


def nearest(points, queries, chunk=256):
    """For each query: the index of the point at the least squared l2
    distance (the lowest index among equal distances), that distance, and
    the second-least distance (inf when there is one point).  FP64."""
    p = np.asarray(points, dtype=np.float64)
    q = np.asarray(queries, dtype=np.float64)
    if p.ndim != 2 or q.ndim != 2 or p.shape[1] != q.shape[1] or p.shape[0] == 0:
        raise ValueError("points [M, D] with M > 0 and queries [N, D]")
    n = q.shape[0]
    idx = np.zeros(n, dtype=np.int64)
    d1 = np.zeros(n)
    d2 = np.full(n, np.inf)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        diff = q[a:b, None, :] - p[None, :, :]
        d = np.einsum("nmd,nmd->nm", diff, diff)
        i = np.argmin(d, axis=1)  # first minimum: the lowest index on ties
        idx[a:b] = i
        d1[a:b] = d[np.arange(b - a), i]
        if p.shape[0] > 1:
            d[np.arange(b - a), i] = np.inf
            d2[a:b] = d.min(axis=1)
    return idx, d1, d2
