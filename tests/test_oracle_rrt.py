"""Pins for the oracle's RRT-Connect (Sec. III-E): a hand-worked run in an
empty scene, a detour around an obstacle whose every edge is checked by the
oracle's edge test independently, an invalid start, and invariants."""
import numpy as np

import oracle
import vpgen
from oracle.rrt import REACHED, _nearest, _steer, rrt_connect
from robots_small import EMPTY_ENV, env_of, planar2

F = np.float32


def test_nearest_and_steer_rules():
    nodes = np.array([[0, 0], [2, 0], [0, 2], [1, 1]], F)
    i, d2 = _nearest(nodes, 4, np.array([1, 0], F))
    assert i == 0 and d2 == 1.0          # ties with nodes 1 and 3: the lowest index
    q_new, s = _steer(np.array([0, 0], F), np.array([3, 4], F), F(25), 2.0)
    np.testing.assert_allclose(q_new, [1.2, 1.6], rtol=1e-6)
    assert s != REACHED
    q_new, s = _steer(np.array([0, 0], F), np.array([0.3, 0.4], F), F(0.25), 2.0)
    assert s == REACHED and np.array_equal(q_new, np.array([0.3, 0.4], F))


def test_empty_scene_one_iteration():
    """Start and goal within range of the first sample: EXTEND(A) reaches
    the sample, CONNECT(B) reaches it too: path start, sample, goal."""
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    start, goal = np.array([0.0, 0.5], F), np.array([0.6, 0.2], F)
    samples = np.array([[0.3, 0.4], [1.0, 1.0]], F)
    solved, iters, path, band, sizes = rrt_connect(o, start, goal, samples, rng=1.0, res=1 / 32, cap=64)
    assert solved == 1 and iters == 1 and not band
    np.testing.assert_array_equal(path, [start, samples[0], goal])
    assert sizes == (2, 2)


def test_detour_around_an_obstacle():
    L1, L2 = 0.7, 0.4
    env = env_of(spheres=[(L1 + L2, 0.0, 0.0, 0.12)])
    o = oracle.Oracle(planar2(L1, L2), env)
    start, goal = np.array([-1.0, 0.0], F), np.array([1.0, 0.0], F)
    assert not o.validate_edges(start[None], goal[None], None, 1 / 32)[0]   # no straight way
    rng = np.random.default_rng(0)
    samples = rng.uniform(-np.pi, np.pi, size=(400, 2)).astype(F)
    solved, iters, path, band, sizes = rrt_connect(o, start, goal, samples, rng=0.5, res=1 / 32, cap=512)
    assert solved == 1 and path.shape[0] >= 3
    np.testing.assert_array_equal(path[0], start)
    np.testing.assert_array_equal(path[-1], goal)
    assert o.validate_edges(path[:-1], path[1:], None, 1 / 32).all()
    steps = np.linalg.norm(path[1:].astype(np.float64) - path[:-1], axis=1)
    assert np.all(steps <= 0.5 + 1e-5)


def test_invalid_start():
    L1, L2 = 0.7, 0.4
    o = oracle.Oracle(planar2(L1, L2), env_of(spheres=[(L1 + L2, 0.0, 0.0, 0.12)]))
    solved, iters, path, band, _ = rrt_connect(o, np.array([0.0, 0.0], F), np.array([1.0, 0.0], F),
                                               np.zeros((5, 2), F), rng=0.5, res=1 / 32, cap=16)
    assert solved == -1 and path is None and iters == 0


def test_arm_problems_give_valid_paths():
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=8)
    o = oracle.Oracle(w.robot, w.env)
    starts, goals = vpgen.uniform_edges(w.robot, 6, seed=5)
    samples = vpgen.uniform_configs(w.robot, 300, seed=6)
    for b in range(6):
        solved, iters, path, band, sizes = rrt_connect(o, starts[b], goals[b], samples, rng=1.0,
                                                       res=float(w.res), cap=400)
        if solved == 1:
            assert o.validate_edges(path[:-1], path[1:], None, float(w.res)).all() or band
            np.testing.assert_array_equal(path[0], starts[b])
            np.testing.assert_array_equal(path[-1], goals[b])
