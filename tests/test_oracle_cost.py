"""Pins for the oracle's penetration cost and gradient, an addition beside
arXiv 2309.14545 (no passage of the paper defines it):
c(q) = sum_s sum_o max(0, r_s + m - d(c_s, o))^2.  Expected values come from
closed forms (a planar arm's Jacobian) and FP64 central finite differences."""
import numpy as np
import pytest

import oracle
import vpgen
from robots_small import env_of, planar2


def test_single_pair_closed_form():
    """Tip sphere of a planar 2-link arm against one obstacle sphere:
    c = (r + m - (|x(q) - p| - rho))^2 with x(q) from the closed form and
    dc/dq = -2 pen (x - p)/|x - p| . dx/dq (planar Jacobian)."""
    L1, L2, r, m = 0.7, 0.4, 0.05, 0.02
    p, rho = np.array([0.9, 0.5, 0.0]), 0.3
    rob = planar2(L1, L2, r)
    rob.sphere_link = rob.sphere_link[1:]
    rob.sphere_centre = rob.sphere_centre[1:]
    rob.sphere_radius = rob.sphere_radius[1:]
    o = oracle.Oracle(rob, env_of(spheres=[(*p, rho)]))
    rng = np.random.default_rng(0)
    hits = 0
    for _ in range(200):
        q1, q2 = rng.uniform(-np.pi, np.pi, size=2)
        x = np.array([L1 * np.cos(q1) + L2 * np.cos(q1 + q2), L1 * np.sin(q1) + L2 * np.sin(q1 + q2), 0.0])
        J = np.array([[-L1 * np.sin(q1) - L2 * np.sin(q1 + q2), -L2 * np.sin(q1 + q2)],
                      [L1 * np.cos(q1) + L2 * np.cos(q1 + q2), L2 * np.cos(q1 + q2)],
                      [0.0, 0.0]])
        n = np.linalg.norm(x - p)
        pen = r + m - (n - rho)
        want_c = max(pen, 0.0) ** 2
        want_g = -2 * max(pen, 0.0) * ((x - p) / n) @ J
        c, g = o.cost(np.array([[q1, q2]]), m)
        assert c[0] == pytest.approx(want_c, abs=1e-13)
        np.testing.assert_allclose(g[0], want_g, atol=1e-12)
        hits += pen > 0
    assert 10 < hits < 190


def test_cost_zero_when_clear():
    rob = planar2()
    o = oracle.Oracle(rob, env_of(spheres=[(5, 5, 5, 0.1)]))
    c, g = o.cost(np.array([[0.3, -0.2]]), 0.02)
    assert c[0] == 0.0 and np.all(g == 0.0)


def _fd(o, q, m, h):
    D = q.shape[0]
    Q = np.repeat(q[None], 2 * D, axis=0)
    for j in range(D):
        Q[2 * j, j] += h
        Q[2 * j + 1, j] -= h
    c = o.cost(Q, m, grad=False)
    return (c[0::2] - c[1::2]) / (2 * h)


@pytest.mark.parametrize("name", [vpgen.ARM7_MIXED128, vpgen.TORSO8_OBB60_CAP20])
def test_gradient_matches_central_differences(name):
    """Central FD in FP64 with h = 1e-6; samples within reach of a kink of the
    distance (FD at h and 2h disagree) are skipped and counted."""
    w = vpgen.workload(name, n_edges=256)
    o = oracle.Oracle(w.robot, w.env)
    m = 0.02
    q = w.q0.astype(np.float64)
    c, g = o.cost(q, m)
    checked = skipped = 0
    for i in range(q.shape[0]):
        if c[i] == 0.0:
            continue
        f1 = _fd(o, q[i], m, 1e-6)
        f2 = _fd(o, q[i], m, 2e-6)
        scale = max(1.0, np.abs(f1).max())
        if np.abs(f1 - f2).max() > 1e-6 * scale:
            skipped += 1
            continue
        assert np.abs(g[i] - f1).max() <= 1e-6 * scale, (i, g[i], f1)
        checked += 1
    assert checked >= 50 and skipped <= 0.05 * (checked + skipped)


def test_gradient_on_a_branching_tree_matches_central_differences():
    """A tree (two branches off joint 1, a second root at joint 6) with
    general origin rotations, general axes and prismatic joints: the oracle's
    Jacobian loop must follow each joint's subtree, which a serial chain does
    not exercise.  Central FD in FP64, kink samples skipped and counted."""
    from robots_small import random_chain
    rng = np.random.default_rng(21)
    r = random_chain(rng, D=9, n_spheres=40)
    r.joint_parent = np.array([-1, 0, 1, 2, 1, 4, -1, 6, 3], dtype=np.int32)
    env = env_of(spheres=[(0.1, 0.0, 0.2, 0.3), (-0.2, 0.3, 0.1, 0.25)],
                 capsules=[(0.0, -0.3, 0.0, 0.3, 0.2, 0.3, 0.08)],
                 cuboids=[(0.2, 0.2, -0.1, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0.15, 0.2, 0.1)])
    o = oracle.Oracle(r, env)
    m = 0.02
    q = rng.uniform(-2.0, 2.0, size=(200, 9))
    c, g = o.cost(q, m)
    checked = skipped = 0
    for i in range(q.shape[0]):
        if c[i] == 0.0:
            continue
        f1 = _fd(o, q[i], m, 1e-6)
        f2 = _fd(o, q[i], m, 2e-6)
        scale = max(1.0, np.abs(f1).max())
        if np.abs(f1 - f2).max() > 1e-6 * scale:
            skipped += 1
            continue
        assert np.abs(g[i] - f1).max() <= 1e-6 * scale, (i, g[i], f1)
        checked += 1
    assert checked >= 50 and skipped <= 0.1 * (checked + skipped)
