"""Pins for the oracle's nearest neighbours (Sec. III-E: l2 distance in a
Euclidean configuration space).  Expected values come from scipy's k-d tree,
hand-computed cases and invariants, never from the oracle itself."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle.nn import nearest


@pytest.mark.parametrize("M,N,D", [(1, 5, 3), (2, 7, 1), (500, 300, 7), (2000, 64, 14), (97, 33, 16)])
def test_matches_kd_tree(M, N, D):
    rng = np.random.default_rng(M + N + D)
    p = rng.uniform(-3, 3, size=(M, D))
    q = rng.uniform(-3, 3, size=(N, D))
    idx, d1, d2 = nearest(p, q)
    dist, j = cKDTree(p).query(q, k=min(2, M))
    if M == 1:
        dist, j = dist[:, None], j[:, None]
    np.testing.assert_allclose(d1, dist[:, 0] ** 2, rtol=1e-12, atol=1e-14)
    assert np.array_equal(idx, j[:, 0])  # random data: no ties
    if M > 1:
        np.testing.assert_allclose(d2, dist[:, 1] ** 2, rtol=1e-12, atol=1e-14)
    else:
        assert np.all(np.isinf(d2))


def test_hand_cases_and_ties():
    p = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 2.0], [2.0, 0.0]])
    q = np.array([[1.0, 0.0],    # equidistant from points 0, 1 and 3: lowest index wins
                  [2.1, 0.0],    # nearest: point 1 (point 3 is a duplicate with a higher index)
                  [0.0, 1.5]])   # nearest: point 2
    idx, d1, d2 = nearest(p, q)
    assert list(idx) == [0, 1, 2]
    np.testing.assert_allclose(d1, [1.0, 0.01, 0.25])
    np.testing.assert_allclose(d2, [1.0, 0.01, 2.25])


def test_invariant_under_translation_and_point_order():
    rng = np.random.default_rng(5)
    p = rng.normal(size=(300, 6))
    q = rng.normal(size=(40, 6))
    idx, d1, _ = nearest(p, q)
    t = rng.normal(size=6)
    idx_t, d1_t, _ = nearest(p + t, q + t)
    assert np.array_equal(idx, idx_t)
    np.testing.assert_allclose(d1, d1_t, rtol=1e-9)
    perm = rng.permutation(300)
    idx_p, d1_p, _ = nearest(p[perm], q)
    assert np.array_equal(perm[idx_p], idx)
    np.testing.assert_allclose(d1_p, d1, rtol=0, atol=0)


def test_query_on_a_point_has_distance_zero():
    rng = np.random.default_rng(8)
    p = rng.normal(size=(50, 7))
    idx, d1, _ = nearest(p, p[[3, 17, 49]])
    assert list(idx) == [3, 17, 49] and np.all(d1 == 0.0)
