"""Pins for the oracle's signed distances and state clearance (Sec.
"Vectorized Collision Checking" of arXiv 2309.14545: robot spheres against
sphere, capsule and cuboid primitives, plus robot self pairs).  Expected
values come from closed forms, special cases and brute-force surface
sampling."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from robots_small import EMPTY_ENV, cuboid_row, env_of, one_joint, planar2

O = oracle.Oracle(planar2(), EMPTY_ENV)  # any instance exposes the distance functions


def test_sphere_distance_closed_form():
    assert O.dist_sphere((3, 4, 0), (0, 0, 0, 1)) == pytest.approx(4.0, abs=1e-15)
    assert O.dist_sphere((0.5, 0, 0), (0, 0, 0, 2)) == pytest.approx(-1.5, abs=1e-15)
    assert O.dist_sphere((1, 1, 1), (1, 1, 1, 0.25)) == pytest.approx(-0.25, abs=1e-15)


def test_capsule_special_cases():
    cap = (0, 0, 0, 2, 0, 0, 0.5)
    assert O.dist_capsule((1, 3, 0), cap) == pytest.approx(2.5, abs=1e-15)       # beside the axis
    assert O.dist_capsule((-3, 4, 0), cap) == pytest.approx(4.5, abs=1e-15)      # beyond p0: distance to p0
    assert O.dist_capsule((5, 0, 4), cap) == pytest.approx(4.5, abs=1e-15)       # beyond p1
    assert O.dist_capsule((1, 0.2, 0), cap) == pytest.approx(-0.3, abs=1e-15)    # inside
    # a point segment is a sphere
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = rng.normal(size=3)
        c = rng.normal(size=3)
        assert O.dist_capsule(x, (*c, *c, 0.3)) == pytest.approx(O.dist_sphere(x, (*c, 0.3)), abs=1e-14)


def test_cuboid_axis_aligned_cases():
    box = cuboid_row((0, 0, 0), np.eye(3), (1, 2, 3))
    assert O.dist_cuboid((0, 0, 0), box) == pytest.approx(-1.0, abs=1e-15)     # centre: nearest face x
    assert O.dist_cuboid((0.5, 1.9, 0), box) == pytest.approx(-0.1, abs=1e-15)  # near the y face
    assert O.dist_cuboid((3, 0, 0), box) == pytest.approx(2.0, abs=1e-15)       # outside along x
    assert O.dist_cuboid((1, 0, 0), box) == pytest.approx(0.0, abs=1e-15)       # on a face
    assert O.dist_cuboid((4, 6, 3), box) == pytest.approx(5.0, abs=1e-15)       # edge region: (3,4,0)
    assert O.dist_cuboid((2, 4, 5), box) == pytest.approx(3.0, abs=1e-15)       # corner: (1,2,2)


def test_cuboid_rotation_covariance():
    """Moving the point and the box by the same rigid motion keeps the distance."""
    rng = np.random.default_rng(1)
    h = np.array([0.3, 0.5, 0.2])
    for _ in range(100):
        x = rng.normal(size=3)
        R = Rotation.from_rotvec(rng.normal(size=3)).as_matrix()
        t = rng.normal(size=3)
        d_aligned = O.dist_cuboid(x, cuboid_row((0, 0, 0), np.eye(3), h))
        d_moved = O.dist_cuboid(R @ x + t, cuboid_row(t, R, h))
        assert d_moved == pytest.approx(d_aligned, abs=1e-13)


def _box_surface(h, n):
    """Dense grid on the six faces of an axis-aligned box of half-extents h."""
    pts = []
    g = np.linspace(-1, 1, n)
    A, B = np.meshgrid(g, g)
    A, B = A.ravel(), B.ravel()
    for ax in range(3):
        o1, o2 = [i for i in range(3) if i != ax]
        for s in (-1, 1):
            p = np.zeros((A.size, 3))
            p[:, ax] = s * h[ax]
            p[:, o1] = A * h[o1]
            p[:, o2] = B * h[o2]
            pts.append(p)
    return np.concatenate(pts)


def _capsule_surface(p0, p1, r, n):
    """Dense samples of a capsule surface: cylinder side plus two hemispheres."""
    u = p1 - p0
    L = np.linalg.norm(u)
    a = u / L
    e1 = np.cross(a, [1, 0, 0] if abs(a[0]) < 0.9 else [0, 1, 0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    th = np.linspace(0, 2 * np.pi, n, endpoint=False)
    s = np.linspace(0, 1, n)
    T, S = np.meshgrid(th, s)
    side = p0 + S.ravel()[:, None] * u + r * (np.cos(T.ravel())[:, None] * e1 + np.sin(T.ravel())[:, None] * e2)
    v = np.random.default_rng(0).normal(size=(n * n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    caps = np.concatenate([p0 + r * v[(v @ a) <= 0], p1 + r * v[(v @ a) >= 0]])
    return np.concatenate([side, caps])


def test_cuboid_brute_force_surface_distance():
    """|d| equals the distance to the nearest surface point (sign: inside < 0),
    within the sampling error of a dense surface grid."""
    rng = np.random.default_rng(2)
    h = np.array([0.25, 0.4, 0.15])
    surf = _box_surface(h, 161)
    spacing = 2 * h.max() / 160
    for _ in range(60):
        x = rng.uniform(-0.8, 0.8, size=3)
        brute = np.linalg.norm(surf - x, axis=1).min()
        inside = np.all(np.abs(x) <= h)
        d = O.dist_cuboid(x, cuboid_row((0, 0, 0), np.eye(3), h))
        assert (d < 0) == inside
        assert abs(abs(d) - brute) <= spacing


def test_capsule_brute_force_surface_distance():
    rng = np.random.default_rng(3)
    p0, p1, r = np.array([0.1, -0.2, 0.3]), np.array([0.5, 0.3, -0.1]), 0.12
    surf = _capsule_surface(p0, p1, r, 400)
    for _ in range(60):
        x = rng.uniform(-0.6, 1.0, size=3)
        brute = np.linalg.norm(surf - x, axis=1).min()
        d = O.dist_capsule(x, (*p0, *p1, r))
        assert abs(abs(d) - brute) <= 4e-3


def test_clearance_is_min_over_terms():
    """K(q) = min over spheres x primitives of d - r_s and over pairs of
    |c_a - c_b| - r_a - r_b; contact (K = 0) counts as valid."""
    # one fixed sphere of radius 0.05 at (0.1, 0.2, 0.3) on the base link,
    # one moving sphere; obstacles at known distances from the fixed one
    rob = one_joint(0, (0, 0, 1), local=(1.0, 0.0, 0.0), r=0.05)
    env = env_of(spheres=[(0.1, 0.2, 0.8, 0.2)], cuboids=[cuboid_row((0.1, -0.5, 0.3), np.eye(3), (0.1, 0.1, 0.1))])
    o = oracle.Oracle(rob, env)
    # q = pi/2 moves the joint sphere to (0, 1, 0), far from both obstacles
    K = o.clearance(np.array([[np.pi / 2]]))[0]
    # base sphere vs sphere: 0.5 - 0.2 - 0.05 = 0.25; vs box: 0.7 - 0.1 - 0.05 = 0.55
    assert K == pytest.approx(0.25, abs=1e-12)
    rob.self_pairs = np.array([[0, 1]], dtype=np.int32)
    o = oracle.Oracle(rob, env)
    # q = 0: joint sphere at (1, 0, 0); pair distance |(0.9,-0.2,-0.3)| - 0.1
    want = min(0.25, np.linalg.norm([0.9, -0.2, -0.3]) - 0.1)
    assert o.clearance(np.array([[0.0]]))[0] == pytest.approx(want, abs=1e-12)
    # touching exactly: a sphere obstacle tangent to the base sphere
    env_t = env_of(spheres=[(0.1, 0.2, 0.5, 0.15)])
    o = oracle.Oracle(one_joint(0, (0, 0, 1), local=(1.0, 0.0, 0.0), r=0.05), env_t)
    assert o.clearance(np.array([[np.pi / 2]]))[0] == pytest.approx(0.0, abs=1e-15)


def test_clearance_takes_each_kind_of_term():
    """Scenes where each kind of term is the binding minimum, with the value
    from a closed form: a self pair (both radii), a capsule beyond its end
    cap, and a rotated cuboid above a face.  One fixed sphere of radius 0.05
    at (0.1, 0.2, 0.3) on the base link; a moving sphere at (cos q, sin q, 0)."""
    rob = one_joint(0, (0, 0, 1), local=(1.0, 0.0, 0.0), r=0.05)
    base = np.array([0.1, 0.2, 0.3])
    rob.self_pairs = np.array([[0, 1]], dtype=np.int32)
    o = oracle.Oracle(rob, EMPTY_ENV)
    for q in np.linspace(-3.0, 3.0, 13):
        moving = np.array([np.cos(q), np.sin(q), 0.0])
        want = np.linalg.norm(moving - base) - 0.05 - 0.05
        assert o.clearance(np.array([[q]]))[0] == pytest.approx(want, abs=1e-12)
    rob.self_pairs = np.zeros((0, 2), dtype=np.int32)
    # capsule along z from 0.6 to 1.6 above the fixed sphere, radius 0.1: the
    # nearest point is the end p0, 0.3 away
    o = oracle.Oracle(rob, env_of(capsules=[(0.1, 0.2, 0.6, 0.1, 0.2, 1.6, 0.1)]))
    assert o.clearance(np.array([[np.pi]]))[0] == pytest.approx(0.3 - 0.1 - 0.05, abs=1e-12)
    # cuboid yawed by 30 degrees about z, its top face 0.3 below the fixed
    # sphere's centre (the face's normal is z, so the yaw leaves the distance)
    R = Rotation.from_euler("z", 30, degrees=True).as_matrix()
    o = oracle.Oracle(rob, env_of(cuboids=[cuboid_row((0.1, 0.2, -0.1), R, (0.1, 0.1, 0.1))]))
    assert o.clearance(np.array([[np.pi]]))[0] == pytest.approx(0.3 - 0.05, abs=1e-12)


def test_exact_contact_is_valid():
    """Contact is allowed (K = 0 is valid), decided on a scene whose
    clearance is exactly 0 in binary floating point: a base sphere of radius
    0.25 at z = 0.5 and an obstacle of radius 0.75 at z = 1.5."""
    import vpgen
    rob = one_joint(0, (0, 0, 1), local=(1.0, 0.0, 0.0), r=0.25)
    rob.sphere_centre = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.5]])
    rob.sphere_radius = np.array([0.05, 0.25])
    o = oracle.Oracle(rob, env_of(spheres=[(0.0, 0.0, 1.5, 0.75)]))
    q = np.array([[np.float32(np.pi / 2)]], dtype=np.float32)
    assert o.clearance(q.astype(np.float64))[0] == 0.0
    assert o.validate_edges(q, q, None, vpgen.RESOLUTION)[0] == 1
    # a hair closer collides
    o = oracle.Oracle(rob, env_of(spheres=[(0.0, 0.0, np.nextafter(1.5, 0.0), 0.75)]))
    assert o.validate_edges(q, q, None, vpgen.RESOLUTION)[0] == 0


def test_non_finite_state_is_invalid():
    o = oracle.Oracle(planar2(), EMPTY_ENV)
    K = o.clearance(np.array([[np.nan, 0.0], [0.0, np.inf], [0.1, 0.2]]))
    assert K[0] == -np.inf and K[1] == -np.inf and K[2] == np.inf
