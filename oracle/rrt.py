"""RRT-Connect on the FP64 oracle -- TEST INFRASTRUCTURE ONLY (see the
package header).

Sec. III-E ("Bringing it Together") names RRT-Connect (Kuffner and LaValle)
as one of the two planners built on the vectorized primitives.  This is the
algorithm's plain form for one problem, batched over problems by the
caller, with the random configurations passed in:

    trees A (rooted at the start) and B (at the goal); for each sample:
        EXTEND(A, sample); if it did not get trapped, CONNECT(B, new node):
        extend B toward it until it is reached (solved) or B is trapped;
        then swap A and B.
    EXTEND(T, q): the node nearest q (l2); step toward q by at most
        `range`; if the edge nearest -> new is valid (every state at the
        resolution, Sec. III-D), add the new node: REACHED if it is q,
        ADVANCED otherwise; else TRAPPED.

The arithmetic that decides which node is nearest and where a new node lies
is float32 with every operation rounded on its own (products, sums,
differences, one square root and one division), so the GPU, doing the same
operations, builds the same trees whenever the edge verdicts agree.  Edge
verdicts come from the FP64 check; an edge inside the clearance band is
flagged (the GPU's FP32 check may decide it otherwise).
"""
from __future__ import annotations

import numpy as np

TRAPPED, ADVANCED, REACHED = 0, 1, 2
F = np.float32


def _nearest(nodes, n, q):
    """Index of the nearest of nodes[:n] to q: squared distance summed in
    coordinate order, each product and sum rounded to float32; the lowest
    index among equal distances."""
    t = nodes[:n] - q[None, :]          # float32, rounded
    acc = np.zeros(n, dtype=F)
    for d in range(q.shape[0]):
        acc = acc + t[:, d] * t[:, d]     # product, then sum, each rounded
    i = int(np.argmin(acc))
    return i, acc[i]


def _steer(near, q, d2, rng):
    """(new node, REACHED or ADVANCED): q itself when within `rng`, else the
    point `rng` away from near along near -> q."""
    dist = np.sqrt(F(d2), dtype=F)
    if dist <= F(rng):
        return q.copy(), REACHED
    s = F(rng) / dist
    return near + s * (q - near), ADVANCED  # float32: difference, product, sum


class _Tree:
    def __init__(self, root, cap):
        self.nodes = np.zeros((cap, root.shape[0]), dtype=F)
        self.parent = np.full(cap, -1, dtype=np.int64)
        self.nodes[0] = root
        self.n = 1


def _extend(o, tree, q, rng, res, band):
    i, d2 = _nearest(tree.nodes, tree.n, q)
    near = tree.nodes[i]
    if d2 == F(0):
        return REACHED, i
    q_new, status = _steer(near, q, d2, rng)
    if tree.n == tree.nodes.shape[0]:
        return TRAPPED, -1
    cls, _ = o.classify_edges(near[None], q_new[None], None, res)
    band[0] |= cls[0] == 2
    if not o.validate_edges(near[None], q_new[None], None, res)[0]:
        return TRAPPED, -1
    tree.nodes[tree.n] = q_new
    tree.parent[tree.n] = i
    tree.n += 1
    return status, tree.n - 1


def _branch(tree, i):
    out = []
    while i >= 0:
        out.append(tree.nodes[i])
        i = tree.parent[i]
    return out  # node i first, root last


def rrt_connect(o, start, goal, samples, rng, res, cap):
    """One problem.  Returns (solved, iterations used, path [n, D] float32
    or None, band flag, tree sizes).  The start and goal must be valid
    states (else solved is -1 and nothing is grown)."""
    start = np.asarray(start, dtype=F)
    goal = np.asarray(goal, dtype=F)
    k = o.clearance(np.stack([start, goal]).astype(np.float64))
    band = [bool(np.any(np.abs(k) <= 1e-4))]
    if np.any(k < 0):
        return -1, 0, None, band[0], (1, 1)
    trees = [_Tree(start, cap), _Tree(goal, cap)]
    a = 0
    for it in range(samples.shape[0]):
        q = np.asarray(samples[it], dtype=F)
        s, i_new = _extend(o, trees[a], q, rng, res, band)
        if s != TRAPPED:
            target = trees[a].nodes[i_new]
            while True:
                sc, j = _extend(o, trees[1 - a], target, rng, res, band)
                if sc != ADVANCED:
                    break
            if sc == REACHED:
                pa = _branch(trees[a], i_new)          # new node ... root of A
                pb = _branch(trees[1 - a], j)          # meeting node ... root of B
                if a == 0:
                    path = pa[::-1] + pb[1:]           # start ... meet ... goal
                else:
                    path = pb[::-1] + pa[1:]
                return 1, it + 1, np.array(path, dtype=F), band[0], (trees[0].n, trees[1].n)
        a = 1 - a
    return 0, samples.shape[0], None, band[0], (trees[0].n, trees[1].n)
