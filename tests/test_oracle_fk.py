"""Pins for the oracle's forward kinematics (Sec. "Vectorized Forward
Kinematics" of arXiv 2309.14545: link poses composed joint by joint; only
sphere positions are produced).  Every expected value here comes from a
closed form, scipy's rotation routines or an invariant, never from the
oracle itself."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import vpgen
from robots_small import EMPTY_ENV, one_joint, planar2, random_chain


def test_planar_two_link_closed_form():
    """x = L1 cos q1 + L2 cos(q1+q2), y = L1 sin q1 + L2 sin(q1+q2)."""
    L1, L2 = 0.7, 0.4
    o = oracle.Oracle(planar2(L1, L2), EMPTY_ENV)
    rng = np.random.default_rng(0)
    q = rng.uniform(-np.pi, np.pi, size=(200, 2))
    c = o.fk(q)
    q1, q2 = q[:, 0], q[:, 1]
    elbow = np.stack([L1 * np.cos(q1), L1 * np.sin(q1), 0 * q1], 1)
    tip = np.stack([L1 * np.cos(q1) + L2 * np.cos(q1 + q2), L1 * np.sin(q1) + L2 * np.sin(q1 + q2), 0 * q1], 1)
    np.testing.assert_allclose(c[:, 0], elbow, atol=1e-12)
    np.testing.assert_allclose(c[:, 1], tip, atol=1e-12)


@pytest.mark.parametrize("make", [lambda: vpgen.arm7(0, 40), lambda: vpgen.torso_arm8(1, 100, 200),
                                  lambda: vpgen.dual_arm14(60, 400)])
def test_rest_pose_is_straight(make):
    """At q = 0 every generated chain stands straight up, so each sphere sits at
    the base offset plus the cumulative link offsets (the generator records
    these positions while it places the spheres)."""
    r = make()
    o = oracle.Oracle(r, EMPTY_ENV)
    c = o.fk(np.zeros((1, r.dof)))[0]
    np.testing.assert_allclose(c, r.rest_world, atol=1e-12)


@pytest.mark.parametrize("axis", [(0, 0, 1), (0, 1, 0), (1, 0, 0), (0.48, -0.6, 0.64)])
def test_single_revolute_matches_scipy(axis):
    """One revolute joint with a fixed origin [R0|t0]: c = t0 + R0 Rot(a, q) p."""
    a = np.array(axis, float)
    a /= np.linalg.norm(a)
    R0 = Rotation.from_euler("xyz", [0.3, -0.7, 1.1]).as_matrix()
    t0 = np.array([0.2, -0.1, 0.4])
    local = np.array([0.3, -0.2, 0.5])
    o = oracle.Oracle(one_joint(vpgen.REVOLUTE, a, R0, t0, local), EMPTY_ENV)
    for q in np.linspace(-3, 3, 13):
        c = o.fk(np.array([[q]]))[0]
        want = t0 + R0 @ Rotation.from_rotvec(a * q).apply(local)
        np.testing.assert_allclose(c[0], want, atol=1e-12)
        np.testing.assert_allclose(c[1], (0.1, 0.2, 0.3), atol=0)  # base-link sphere never moves


def test_single_prismatic_is_translation():
    a = np.array([0.6, 0.0, 0.8])
    R0 = Rotation.from_euler("z", 0.5).as_matrix()
    t0 = np.array([0.1, 0.2, 0.3])
    local = np.array([0.3, -0.2, 0.5])
    o = oracle.Oracle(one_joint(vpgen.PRISMATIC, a, R0, t0, local), EMPTY_ENV)
    for q in (-0.4, 0.0, 0.25, 1.0):
        c = o.fk(np.array([[q]]))[0]
        np.testing.assert_allclose(c[0], t0 + R0 @ (a * q + local), atol=1e-12)


@pytest.mark.parametrize("parents", [None, [-1, 0, 1, 2, 1, 4, -1, 6, 3]])
def test_random_chain_matches_scipy_composition(parents):
    """General chain, and a tree (two branches off joint 1, a second root at
    joint 6): compose the frames with scipy rotations, independently."""
    rng = np.random.default_rng(3)
    r = random_chain(rng, D=6 if parents is None else len(parents), n_spheres=15)
    if parents is not None:
        r.joint_parent = np.array(parents, dtype=np.int32)
    o = oracle.Oracle(r, EMPTY_ENV)
    for _ in range(20):
        q = rng.uniform(-2, 2, size=r.dof)
        Rs, ts = [np.eye(3)], [np.zeros(3)]
        for j in range(r.dof):
            Rp, tp = Rs[r.joint_parent[j] + 1], ts[r.joint_parent[j] + 1]
            F = r.joint_origin[j]
            RJ, tJ = Rp @ F[:, :3], tp + Rp @ F[:, 3]
            if r.joint_type[j] == vpgen.REVOLUTE:
                Rs.append(RJ @ Rotation.from_rotvec(r.joint_axis[j] * q[j]).as_matrix())
                ts.append(tJ)
            else:
                Rs.append(RJ)
                ts.append(tJ + RJ @ (r.joint_axis[j] * q[j]))
        want = np.array([ts[l] + Rs[l] @ p for l, p in zip(r.sphere_link, r.sphere_centre)])
        np.testing.assert_allclose(o.fk(q[None])[0], want, atol=1e-12)
        frames = o.link_frames(q)
        for l in range(r.dof + 1):
            np.testing.assert_allclose(frames[l][:, :3], Rs[l], atol=1e-12)
            np.testing.assert_allclose(frames[l][:, 3], ts[l], atol=1e-12)


@pytest.mark.parametrize("name", [vpgen.ARM7_SPHERES16, vpgen.TORSO8_OBB60_CAP20, vpgen.DUAL14_SHELVES])
def test_frames_orthonormal_and_rigid_links(name):
    """Invariants: every link rotation is orthonormal with det +1, and
    distances between spheres on one link do not depend on q."""
    r = vpgen.robot_for(name)
    o = oracle.Oracle(r, EMPTY_ENV)
    q = vpgen.uniform_configs(r, 32, seed=11).astype(np.float64)
    c0 = o.fk(np.zeros((1, r.dof)))[0]
    c = o.fk(q)
    for i in range(q.shape[0]):
        F = o.link_frames(q[i])
        for l in range(r.n_links):
            R = F[l][:, :3]
            assert np.abs(R.T @ R - np.eye(3)).max() < 1e-12
            assert abs(np.linalg.det(R) - 1.0) < 1e-12
    for l in range(r.n_links):
        idx = np.nonzero(r.sphere_link == l)[0]
        if len(idx) < 2:
            continue
        d0 = np.linalg.norm(c0[idx, None] - c0[None, idx], axis=-1)
        d = np.linalg.norm(c[:, idx, None] - c[:, None, idx], axis=-1)
        assert np.abs(d - d0).max() < 1e-12
