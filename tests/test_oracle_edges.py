"""Pins for the oracle's edge validation (Sec. "Vectorized Motion Validation"
of arXiv 2309.14545: an edge is valid iff every state of its discretisation
is valid; Sec. "Bringing it Together": linear interpolation in a Euclidean
C-space).  Expected values are hand-computed counts, brute force over the
states, and subset relations between discretisations."""
import numpy as np
import pytest

import oracle
import vpgen
from robots_small import EMPTY_ENV, planar2

RES = np.float32(1.0 / 32.0)


def _count(o, a, b, res=RES):
    return int(o.edge_count(np.array([a], np.float32), np.array([b], np.float32), res)[0])


def test_edge_count_hand_cases():
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    assert _count(o, [0, 0], [0, 0]) == 2                       # constant edge: both endpoints
    assert _count(o, [0, 0], [1.0, 0.2]) == 33                  # 32 steps of 1/32 rad
    assert _count(o, [0, 0], [0.5, -0.1]) == 17
    assert _count(o, [0, 0], [1 / 32, 0]) == 2                  # exactly one step
    step_plus = np.nextafter(np.float32(1 / 32), np.float32(1))
    assert _count(o, [0, 0], [step_plus, 0]) == 3               # a hair over one step
    assert _count(o, [0.3, -2.8], [0.3, 2.8]) == 181            # ceil(5.6 * 32) + 1
    assert _count(o, [0, 0], [0.5, 0], res=np.float32(0.1)) == 6


def test_edge_count_is_decided_in_float32():
    """The count is an integer decided in float32, the precision the method
    runs in: q1 - q0 = 1 + 1e-8 rounds to 1.0f, so k = 33 (float64 would
    give ceil(32.0000003) + 1 = 34)."""
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    assert _count(o, [np.float32(-1e-8), 0], [1.0, 0]) == 33


def test_edge_count_division_is_float32():
    """The quotient is a float32 division too: 0.3f / 0.1f is exactly
    3.0000000745... (checked with exact rationals), which float32 rounds to
    3.0, so k = 3 + 1; exact or float64 division would give ceil = 4, k = 5."""
    from fractions import Fraction
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    d, r = np.float32(0.3), np.float32(0.1)
    exact = Fraction(float(d)) / Fraction(float(r))
    assert 3 < exact < Fraction(3) + Fraction(1, 10 ** 7)
    assert _count(o, [0, 0], [d, 0], res=r) == 4


def test_edge_count_non_finite():
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    assert _count(o, [np.nan, 0], [0, 0]) == -1
    assert _count(o, [0, 0], [np.inf, 0]) == -1


def test_edge_states_endpoints_and_spacing():
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    q0 = np.array([0.1, -0.7], np.float32)
    q1 = np.array([1.3, 0.4], np.float32)
    for k in (2, 3, 17, 40):
        s = o.edge_states(q0, q1, k)
        assert np.array_equal(s[0], q0.astype(np.float64))
        assert np.array_equal(s[-1], q1.astype(np.float64))
        np.testing.assert_allclose(np.diff(s, axis=0), (q1.astype(np.float64) - q0)[None] / (k - 1) * np.ones((k - 1, 1)),
                                   atol=1e-15)


def test_denser_grid_contains_the_grid():
    """States of a k-state edge are every 4th state of the 4(k-1)+1-state
    edge (exactly), so validity at 4x density implies validity at k."""
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=300)
    o = oracle.Oracle(w.robot, w.env)
    k = o.edge_count(w.q0, w.q1, w.res)
    for e in range(5):
        a = o.edge_states(w.q0[e], w.q1[e], k[e])
        b = o.edge_states(w.q0[e], w.q1[e], 4 * (k[e] - 1) + 1)
        assert np.array_equal(a, b[::4])
    v = o.validate_edges(w.q0, w.q1, None, w.res)
    v4 = o.validate_edges(w.q0, w.q1, 4 * (k - 1) + 1)
    assert np.all(v[v4 == 1] == 1)
    assert 0 < v.mean() < 1


@pytest.mark.parametrize("name", [vpgen.ARM7_SPHERES16, vpgen.TORSO8_OBB60_CAP20, vpgen.DUAL14_SHELVES])
def test_edge_verdict_is_every_state_valid(name):
    """Brute force: the edge verdict equals 'every state has K >= 0'."""
    w = vpgen.workload(name, n_edges=40)
    o = oracle.Oracle(w.robot, w.env)
    counts = w.counts if w.counts is not None else o.edge_count(w.q0, w.q1, w.res)
    counts = np.minimum(counts, 64)
    v = o.validate_edges(w.q0, w.q1, counts)
    cls, nb = o.classify_edges(w.q0, w.q1, counts)
    for e in range(40):
        K = o.clearance(o.edge_states(w.q0[e], w.q1[e], counts[e]))
        assert v[e] == int(np.all(K >= 0))
        first_bad = np.nonzero(K < -oracle.BAND)[0]
        if first_bad.size:
            assert cls[e] == 1
            assert nb[e] == int(np.sum(np.abs(K[:first_bad[0]]) <= oracle.BAND))
        elif np.any(np.abs(K) <= oracle.BAND):
            assert cls[e] == 2
        else:
            assert cls[e] == 0 and v[e] == 1


def test_two_state_and_constant_edges_reduce_to_state_checks():
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=200)
    o = oracle.Oracle(w.robot, w.env)
    K0 = o.clearance(w.q0.astype(np.float64))
    K1 = o.clearance(w.q1.astype(np.float64))
    v2 = o.validate_edges(w.q0, w.q1, np.full(200, 2, np.int32))
    assert np.array_equal(v2, ((K0 >= 0) & (K1 >= 0)).astype(np.uint8))
    vc = o.validate_edges(w.q0, w.q0, None, w.res)
    assert np.array_equal(vc, (K0 >= 0).astype(np.uint8))


def test_bad_counts_and_non_finite_edges_are_invalid():
    o = oracle.Oracle(planar2(), EMPTY_ENV)  # nothing to hit: every finite state is valid
    q0 = np.array([[0, 0], [0, 0], [np.nan, 0], [0, 0]], np.float32)
    q1 = np.array([[1, 1], [1, 1], [1, 1], [np.inf, 0]], np.float32)
    assert list(o.validate_edges(q0, q1, np.array([5, 1, 5, 5], np.int32))) == [1, 0, 0, 0]
    assert list(o.validate_edges(q0, q1, None, RES)) == [1, 1, 0, 0]
    # counts of 0 or below are invalid too (no state would be checked at all)
    assert list(o.validate_edges(q0[:2], q1[:2], np.array([0, -3], np.int32))) == [0, 0]


def test_over_long_edges_have_no_count():
    """A count above 2^24 steps is refused (-1): 1e7 rad at 1/32 rad would be
    3.2e8 steps.  The largest accepted edge has exactly 2^24 steps."""
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    assert _count(o, [0, 0], [1e7, 0]) == -1
    assert _count(o, [0, 0], [2.0 ** 24 / 32, 0]) == 2 ** 24 + 1
    assert _count(o, [0, 0], [np.nextafter(np.float32(2.0 ** 24 / 32), np.float32(1e9)), 0]) == -1


def test_explicit_counts_past_the_step_limit_are_invalid():
    """An explicit count may be no longer than the longest edge a resolution
    can give (2^24 steps, 2^24 + 1 states): past that the edge is invalid
    without a state being checked, as a count below 2 is.  In an empty scene
    every state is valid, so only the bound can make these edges invalid;
    the count 2^31 - 1 would otherwise take minutes of state checks."""
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    q0 = np.zeros((1, 2), np.float32)
    q1 = np.ones((1, 2), np.float32)
    assert list(o.validate_edges(q0, q1, np.array([2 ** 24 + 2], np.int32))) == [0]
    assert list(o.validate_edges(q0, q1, np.array([2 ** 31 - 1], np.int32))) == [0]
    cls, nb = o.classify_edges(q0, q1, np.array([2 ** 24 + 2], np.int32))
    assert list(cls) == [1] and list(nb) == [0]
    # the longest accepted explicit count still checks its states (2^24 + 1
    # states of a planar arm in an empty scene: a second or two)
    assert list(o.validate_edges(q0, q1, np.array([2 ** 24 + 1], np.int32), n_threads=1)) == [1]
