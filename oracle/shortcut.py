"""Randomized shortcutting on the FP64 oracle -- TEST INFRASTRUCTURE ONLY
(see the package header).

Sec. III-E ("Bringing it Together") lists randomized shortcutting among the
planners' simplification steps: repeatedly pick two points of a path and,
if the straight motion between them is valid, drop what lies between.  The
batched form here runs every path in lockstep, one candidate per path and
step, from random numbers passed in:

* path p with n >= 3 waypoints draws i = floor(u0 n), j = floor(u1 n)
  (products rounded to float32, the method's precision; clamped to n - 1),
  swapped so that i <= j;
* if j - i >= 2, the edge waypoint i -> waypoint j is checked as every
  edge is (Sec. III-D: all states at the resolution), and when valid the
  waypoints strictly between are removed (the rest keep their order).
"""
from __future__ import annotations

import numpy as np


def candidate(u0, u1, n):
    """Waypoint pair (i, j) for one path of n waypoints, or None."""
    if n < 3:
        return None
    nf = np.float32(n)
    i = min(int(np.floor(np.float32(u0) * nf)), n - 1)
    j = min(int(np.floor(np.float32(u1) * nf)), n - 1)
    if i > j:
        i, j = j, i
    return (i, j) if j - i >= 2 else None


def shortcut(o, paths, lengths, draws, res):
    """Returns (paths, lengths, band): the shortened paths (float32, the
    same shape; entries past each length unspecified), their lengths, and a
    per-path flag set when some candidate edge of that path was within the
    clearance band (there the verdict is not pinned and FP32 may decide
    otherwise)."""
    paths = np.array(paths, dtype=np.float32, copy=True)
    lengths = np.array(lengths, dtype=np.int64, copy=True)
    P = paths.shape[0]
    band = np.zeros(P, dtype=bool)
    for t in range(draws.shape[0]):
        cand = []
        for p in range(P):
            c = candidate(draws[t, p, 0], draws[t, p, 1], int(lengths[p]))
            if c is not None:
                cand.append((p,) + c)
        if not cand:
            continue
        q0 = np.stack([paths[p, i] for p, i, j in cand])
        q1 = np.stack([paths[p, j] for p, i, j in cand])
        cls, _ = o.classify_edges(q0, q1, None, res)
        ok = o.validate_edges(q0, q1, None, res)
        for (p, i, j), c, v in zip(cand, cls, ok):
            band[p] |= c == 2
            if v:
                n = int(lengths[p])
                paths[p, i + 1:i + 1 + (n - j)] = paths[p, j:n].copy()
                lengths[p] = n - (j - i - 1)
    return paths, lengths, band
