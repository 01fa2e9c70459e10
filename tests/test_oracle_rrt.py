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


def test_nearest_and_steer_are_float32():
    """Both decisions are float32 with every operation rounded on its own.
    Query (0.1, 0) against nodes (0.5, 0.3) and (0.1, 0.5): in float32 both
    squared distances come to 0.25 exactly, a tie that goes to the lower
    index, while in exact arithmetic node 0 is 0.2500000059... away and node
    1 is nearer.  Steering from 0.1 toward -0.2 by 0.1: the step
    s * (q - near) rounds to exactly -0.1f, so the new node is 0.0, where a
    float64 evaluation would leave 5.96e-9."""
    i, d2 = _nearest(np.array([[0.5, 0.3], [0.1, 0.5]], F), 2, np.array([0.1, 0.0], F))
    assert i == 0 and d2 == F(0.25)
    near, q = np.array([0.1], F), np.array([-0.2], F)
    _, d2 = _nearest(near[None], 1, q)
    q_new, s = _steer(near, q, d2, 0.1)
    assert s != REACHED and q_new[0] == F(0.0)


def test_a_sample_exactly_at_range_is_reached():
    # |q - near| = 0.5 = range exactly: REACHED, the sample itself
    q_new, s = _steer(np.array([0, 0], F), np.array([0.5, 0], F), F(0.25), 0.5)
    assert s == REACHED and np.array_equal(q_new, np.array([0.5, 0], F))


def _slider(obstacle_radius=None):
    """One prismatic joint along x carrying a sphere of radius 0.1; with an
    obstacle sphere at the origin, states with |q| < 0.1 + radius collide."""
    from robots_small import one_joint
    r = one_joint(vpgen.PRISMATIC, (1.0, 0.0, 0.0), local=(0.0, 0.0, 0.0), r=0.1)
    r.sphere_link = np.array([1], dtype=np.int32)
    r.sphere_centre = np.zeros((1, 3))
    r.sphere_radius = np.array([0.1])
    env = EMPTY_ENV if obstacle_radius is None else env_of(spheres=[(0.0, 0.0, 0.0, obstacle_radius)])
    return oracle.Oracle(r, env)


def test_trees_alternate():
    """Start -2, goal 2, the middle (|q| < 0.55) blocked, range 1.5, samples
    -1 then +1.  Sample 1: EXTEND(A) reaches -1; CONNECT(B) steps from 2 to
    0.5, which collides.  The trees swap.  Sample 2: EXTEND(B) reaches +1;
    CONNECT(A) steps from -1 to 0.5 and is trapped.  Unsolved after 2
    samples, with 2 nodes in each tree (without the swap, A would try +1 and
    B would keep its single node)."""
    o = _slider(0.45)
    solved, iters, path, band, sizes = rrt_connect(o, np.array([-2.0], F), np.array([2.0], F),
                                                   np.array([[-1.0], [1.0]], F), rng=1.5, res=1 / 32, cap=16)
    assert solved == 0 and iters == 2 and path is None and not band
    assert sizes == (2, 2)


def test_a_sample_on_a_node_adds_nothing():
    """Empty scene; the first sample is the start itself: EXTEND(A) finds it
    at distance 0 and adds no node; CONNECT(B) then walks from the goal to
    the start in steps of the range: 2 -> 0.5 -> -1 -> -2 (the last within
    range, so the start itself)."""
    o = _slider()
    start, goal = np.array([-2.0], F), np.array([2.0], F)
    solved, iters, path, band, sizes = rrt_connect(o, start, goal, np.array([[-2.0]], F), rng=1.5,
                                                   res=1 / 32, cap=16)
    assert solved == 1 and iters == 1
    assert sizes == (1, 4)
    np.testing.assert_array_equal(path[:, 0], np.array([-2.0, -1.0, 0.5, 2.0], F))


def test_full_trees_are_trapped():
    """Capacity 3 with the middle blocked: samples -1, 1, -1.5, 1.5 fill both
    trees to 3 nodes (each connect is blocked at 0.5 or -0.5); samples -2.5
    and 2.5 then find their tree full and add nothing."""
    o = _slider(0.45)
    samples = np.array([[-1.0], [1.0], [-1.5], [1.5], [-2.5], [2.5]], F)
    solved, iters, path, band, sizes = rrt_connect(o, np.array([-2.0], F), np.array([2.0], F), samples,
                                                   rng=1.5, res=1 / 32, cap=3)
    assert solved == 0 and iters == 6 and path is None
    assert sizes == (3, 3)


def test_invalid_goal_and_band_endpoints():
    o = _slider(0.45)
    # the goal inside the obstacle: nothing is grown
    solved, iters, path, band, sizes = rrt_connect(o, np.array([-2.0], F), np.array([0.2], F),
                                                   np.array([[1.0]], F), rng=1.5, res=1 / 32, cap=8)
    assert solved == -1 and iters == 0 and path is None
    # a start 5e-5 m clear of the obstacle: inside the 1e-4 band, so flagged
    solved, iters, path, band, sizes = rrt_connect(o, np.array([-0.55005], F), np.array([2.0], F),
                                                   np.zeros((0, 1), F), rng=1.5, res=1 / 32, cap=8)
    assert solved == 0 and band


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
