"""The link-level spheres the kernels cull with (Sec. III-D mid-phase), read
back through vp_link_bounds and checked in float64 against the robot's own
spheres.  The verdict tests cannot see a bound that is merely loose, and a
bound that is too small shows there only where it hides a collision; here
every sphere is checked to lie inside its link's sphere and its half's."""
import dataclasses

import numpy as np
import pytest

import vpgen

pytestmark = pytest.mark.gpu

MARGIN = 1e-5  # the float margin the packer adds to every radius


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    return Validator, vp


def _robots():
    from robots_small import random_chain
    rng = np.random.default_rng(11)
    small = random_chain(rng, D=6, n_spheres=30)
    # a link of exactly 4 spheres and one of 3 (split / not split)
    rest = rng.choice([0, 3, 4, 5, 6], size=small.n_spheres - 7)
    small.sphere_link = np.array([1] * 4 + [2] * 3 + list(rest), dtype=np.int32)
    return [vpgen.robot_for(vpgen.ARM7_SPHERES16), vpgen.robot_for(vpgen.TORSO8_OBB60_CAP20),
            vpgen.robot_for(vpgen.DUAL14_SHELVES), small]


def _need(centre, C, R):
    return float(np.max(np.linalg.norm(C - centre, axis=1) + R))


@pytest.mark.parametrize("idx", range(4))
def test_bounds_enclose_their_spheres(vpmod, idx):
    Validator, _ = vpmod
    r = _robots()[idx]
    val = Validator(r, vpgen.Env(np.zeros((0, 4)), np.zeros((0, 7)), np.zeros((0, 15))))
    link, half, which = val.link_bounds()
    L = r.dof + 1
    C = np.asarray(r.sphere_centre, np.float64)
    R = np.asarray(r.sphere_radius, np.float64)
    sl = np.asarray(r.sphere_link)
    for l in range(L):
        m = sl == l
        if not m.any():
            assert link[l, 3] < 0 and (half[l, :, 3] < 0).all()
            continue
        c = link[l, :3].astype(np.float64)
        # encloses every sphere of the link, with the float margin to spare
        assert _need(c, C[m], R[m]) <= float(link[l, 3]) - 0.5 * MARGIN, l
        # never looser than the given sphere or the mean-centre bound
        mean_bound = _need(C[m].mean(0), C[m], R[m])
        assert float(link[l, 3]) <= mean_bound + MARGIN + 1e-6, l
        if r.link_spheres is not None:
            assert float(link[l, 3]) <= float(r.link_spheres[l][3]) + MARGIN + 1e-6, l
        if m.sum() >= 4:
            for h in (0, 1):
                mh = m & (which == h)
                assert mh.sum() >= 2, (l, h)
                ch = half[l, h, :3].astype(np.float64)
                assert _need(ch, C[mh], R[mh]) <= float(half[l, h, 3]) - 0.5 * MARGIN, (l, h)
            assert set(which[m]) == {0, 1}
        else:
            assert (which[m] == -1).all() and (half[l, :, 3] < 0).all()


def test_given_envelopes_are_tightened(vpmod):
    """The torso arm's given link spheres are loose envelopes; the packed
    ones are the packer's own, smaller bounds."""
    Validator, _ = vpmod
    r = vpgen.robot_for(vpgen.TORSO8_OBB60_CAP20)
    val = Validator(r, vpgen.Env(np.zeros((0, 4)), np.zeros((0, 7)), np.zeros((0, 15))))
    link, _, _ = val.link_bounds()
    given = np.asarray(r.link_spheres)[:, 3]
    assert (link[:, 3] < given).all()
    assert link[:, 3].sum() < 0.8 * given.sum()


def test_bounds_errors(vpmod):
    Validator, vp = vpmod
    r = vpgen.robot_for(vpgen.ARM7_SPHERES16)
    val = Validator(r, vpgen.Env(np.zeros((0, 4)), np.zeros((0, 7)), np.zeros((0, 15))))
    with pytest.raises(vp.VPError) as e:
        vp.vp_link_bounds(val.ctx, r.dof, r.n_spheres)
    assert e.value.status == vp.VP_ERR_ARG
    # a given sphere that misses one of its link's spheres is refused on load
    bad = dataclasses.replace(vpgen.robot_for(vpgen.TORSO8_OBB60_CAP20))
    ls = np.array(bad.link_spheres, copy=True)
    ls[3, 3] = 0.01
    bad.link_spheres = ls
    with pytest.raises(vp.VPError) as e:
        Validator(bad, vpgen.Env(np.zeros((0, 4)), np.zeros((0, 7)), np.zeros((0, 15))))
    assert e.value.status == vp.VP_ERR_ARG
