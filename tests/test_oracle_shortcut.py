"""Pins for the oracle's randomized shortcutting (Sec. III-E): hand-worked
draws in an empty scene and against a wall, and invariants (endpoints kept,
the result a subsequence of the input, lengths never grow)."""
import numpy as np

import oracle
import vpgen
from oracle.shortcut import candidate, shortcut
from robots_small import EMPTY_ENV, env_of, planar2


def test_candidate_rule():
    assert candidate(0.1, 0.9, 2) is None            # fewer than 3 waypoints
    assert candidate(0.0, 0.99, 10) == (0, 9)
    assert candidate(0.95, 0.05, 10) == (0, 9)       # swapped
    assert candidate(0.31, 0.42, 10) is None         # j - i = 1: nothing between
    assert candidate(0.999999, 0.0, 5) == (0, 4)
    assert candidate(1.0, 0.0, 5) == (0, 4)          # floor(1 * 5) = 5, clamped to n - 1
    assert candidate(0.0, 1.0, 5) == (0, 4)          # the same for the second draw
    assert candidate(0.7, 0.0, 4) == (0, 2)          # floor(2.8), not its rounding


def test_candidate_product_is_float32():
    """u = 0.45454543828964233 (a float32) times 11 is exactly 4.99999982...
    (checked with rationals), which float32 rounds to 5.0: the waypoint is
    5, where exact or float64 arithmetic would give 4."""
    from fractions import Fraction
    u = np.float32(0.45454543828964233)
    assert Fraction(float(u)) * 11 < 5 and np.float32(u) * np.float32(11) == np.float32(5)
    assert candidate(u, 0.0, 11) == (0, 5)


def test_empty_scene_hand_worked():
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    path = np.stack([np.linspace(0, 1, 8), np.zeros(8)], 1).astype(np.float32)[None]
    draws = np.array([[[0.15, 0.70]], [[0.0, 0.5]]], np.float32)   # (1, 5), then (0, 2) on the shorter path
    out, n, band = shortcut(o, path, np.array([8]), draws, 1.0 / 32)
    # step 1 removes waypoints 2, 3, 4 -> [0, 1, 5, 6, 7]; step 2 removes index 1 -> [0, 5, 6, 7]
    assert n[0] == 4 and not band[0]
    np.testing.assert_array_equal(out[0, :4], path[0, [0, 5, 6, 7]])


def test_wall_blocks_the_shortcut():
    """A planar arm whose tip sweeps through an obstacle sphere at (1.1, 0)
    when the first joint moves straight from -1 to 1 rad.  The detour folds
    the elbow first (q2 = 2.5 keeps the tip within 0.4 m of the elbow, and
    the elbow stays 0.4 m or more from the obstacle), so it is free; the
    shortcut from the first to the last waypoint is not."""
    L1, L2 = 0.7, 0.4
    env = env_of(spheres=[(L1 + L2, 0.0, 0.0, 0.12)])
    o = oracle.Oracle(planar2(L1, L2), env)
    path = np.array([[[-1.0, 0.0], [-1.0, 2.5], [1.0, 2.5], [1.0, 0.0]]], np.float32)
    assert o.validate_edges(path[0, :-1], path[0, 1:], None, 1 / 32).all()      # the detour is free
    assert not o.validate_edges(path[0, :1], path[0, -1:], None, 1 / 32)[0]     # the straight move is not
    out, n, band = shortcut(o, path, np.array([4]), np.array([[[0.0, 0.99]]], np.float32), 1.0 / 32)
    assert n[0] == 4 and not band[0]
    np.testing.assert_array_equal(out, path)


def test_invariants_on_jagged_paths():
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=8)
    o = oracle.Oracle(w.robot, w.env)
    paths = vpgen.jagged_paths(w.robot, 24, 12, seed=3)
    draws = vpgen.shortcut_draws(15, 24, seed=4)
    out, n, band = shortcut(o, paths, np.full(24, 12), draws, float(w.res))
    assert np.all(n <= 12) and np.all(n >= 2) and n.min() < 12
    for p in range(24):
        np.testing.assert_array_equal(out[p, 0], paths[p, 0])
        np.testing.assert_array_equal(out[p, n[p] - 1], paths[p, -1])
        rows = [tuple(r) for r in paths[p]]
        idx = [rows.index(tuple(r)) for r in out[p, :n[p]]]
        assert idx == sorted(idx) and len(set(idx)) == len(idx)   # a subsequence, in order
