"""The seeded workload generator: the obstacle-shifted variants keep the
base workload's robot, edges and counts and move only the obstacles."""
import numpy as np
import pytest

import vpgen


@pytest.mark.parametrize("variant,base,axis,shift", [(vpgen.DUAL14_SHELVES_FAR, vpgen.DUAL14_SHELVES, None, 0.6),
                                                     (vpgen.DUAL14_MIXED1000_FAR, vpgen.DUAL14_MIXED1000, 0, 1.0)])
def test_variant_moves_only_the_obstacles(variant, base, axis, shift):
    v = vpgen.workload(variant, n_edges=5000)
    b = vpgen.workload(base, n_edges=5000)
    assert v.name == variant
    assert np.array_equal(v.q0, b.q0) and np.array_equal(v.q1, b.q1) and np.array_equal(v.counts, b.counts)
    assert v.robot.dof == b.robot.dof and v.env.n_prims == b.env.n_prims
    cv, cb = v.env.cuboids[:, :3], b.env.cuboids[:, :3]
    if axis is None:  # shelf units pushed radially: every board farther from the robot
        assert np.linalg.norm(cv[:, :2], axis=1).mean() > np.linalg.norm(cb[:, :2], axis=1).mean() + 0.5 * shift
    else:  # cube centre moved along x
        for kind in ("spheres", "capsules", "cuboids"):
            pv, pb = getattr(v.env, kind)[:, axis], getattr(b.env, kind)[:, axis]
            assert abs((pv.mean() - pb.mean()) - shift) < 0.15


def test_every_workload_name_resolves():
    for name in vpgen.NAMES:
        w = vpgen.workload(name, n_edges=64)
        assert w.q0.shape == (64, w.robot.dof) and w.name == name


@pytest.mark.parametrize("name,scene", [(vpgen.DUAL14_SHELVES_MID, vpgen.DUAL14_SHELVES),
                                        (vpgen.DUAL14_MIXED1000_MID, vpgen.DUAL14_MIXED1000_FAR)])
def test_mid_variants_draw_endpoints_near_the_middle(name, scene):
    """The mid variants keep their scene (the shelves, or the far cube) and
    draw both endpoints within the middle half of every joint's range, with
    the same log-uniform counts; a prefix equals the full draw's."""
    w = vpgen.workload(name, n_edges=70_000)
    s = vpgen.workload(scene, n_edges=16)
    lo, hi = w.robot.joint_lo, w.robot.joint_hi
    mid, quarter = 0.5 * (lo + hi), 0.25 * (hi - lo)
    for q in (w.q0, w.q1):
        assert np.all(np.abs(q - mid) <= quarter * (1 + 1e-6))
        assert np.all(np.abs(q - mid).max(axis=0) > 0.95 * quarter)
    assert np.array_equal(w.env.cuboids, s.env.cuboids) and np.array_equal(w.env.spheres, s.env.spheres)
    assert w.counts.min() >= 2 and w.counts.max() <= 512
    p = vpgen.workload(name, n_edges=1000)
    assert np.array_equal(p.q0, w.q0[:1000]) and np.array_equal(p.counts, w.counts[:1000])
