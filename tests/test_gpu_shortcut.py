"""Batched randomized shortcutting (vp_shortcut_paths) against the FP64
oracle running the same steps on the same random numbers.  A path whose
every candidate edge was outside the clearance band must come out
identical (same length, bit-identical waypoints); a path with a band
candidate may legitimately differ and is checked for the invariants only."""
import numpy as np
import pytest
import torch

import oracle
import vpgen
from oracle.shortcut import shortcut

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    return Validator, vp


def _invariants(orig, n0, out, n, W):
    """Endpoints kept, lengths only shrink, the result an ordered
    subsequence of each path's original waypoints."""
    for p in range(orig.shape[0]):
        assert 2 <= n[p] <= n0[p] <= W
        np.testing.assert_array_equal(out[p, 0], orig[p, 0])
        np.testing.assert_array_equal(out[p, n[p] - 1], orig[p, n0[p] - 1])
        rows = [tuple(r) for r in orig[p, :n0[p]]]
        idx = [rows.index(tuple(r)) for r in out[p, :n[p]]]
        assert idx == sorted(idx) and len(set(idx)) == len(idx)


@pytest.mark.parametrize("name,P,W,T", [(vpgen.ARM7_SPHERES16, 300, 16, 24), (vpgen.TORSO8_OBB60_CAP20, 200, 12, 12),
                                        (vpgen.DUAL14_SHELVES, 96, 10, 8)])
def test_shortcut_matches_oracle(vpmod, name, P, W, T):
    Validator, vp = vpmod
    w = vpgen.workload(name, n_edges=8)
    paths = vpgen.jagged_paths(w.robot, P, W, seed=17 + W)
    draws = vpgen.shortcut_draws(T, P, seed=19 + T)
    lengths = np.full(P, W, np.int32)
    lengths[:5] = [2, 3, W - 1, W, 1]  # short and ragged paths
    val = Validator(w.robot, w.env)
    gp = torch.from_numpy(paths).cuda()
    gl = torch.from_numpy(lengths).cuda()
    val.shortcut(gp, gl, torch.from_numpy(draws).cuda(), float(w.res))
    got_p, got_n = gp.cpu().numpy(), gl.cpu().numpy()
    want_p, want_n, band = shortcut(oracle.Oracle(w.robot, w.env), paths, lengths, draws, float(w.res))
    pinned = ~band
    assert pinned.mean() > 0.8
    assert np.array_equal(got_n[pinned], want_n[pinned])
    for p in np.nonzero(pinned)[0]:
        np.testing.assert_array_equal(got_p[p, :got_n[p]], want_p[p, :want_n[p]])
    assert got_n[0] == 2 and got_n[4] == 1  # fewer than 3 waypoints: untouched
    ok = lengths >= 2
    _invariants(paths[ok], lengths[ok], got_p[ok], got_n[ok], W)
    assert got_n[ok].mean() < W - 1  # shortcuts were taken
    val.close()


def test_shortcut_edge_cases(vpmod):
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=8)
    val = Validator(w.robot, w.env)
    paths = torch.from_numpy(vpgen.jagged_paths(w.robot, 4, 6, seed=1)).cuda()
    before = paths.clone()
    lengths = torch.full((4,), 6, dtype=torch.int32, device="cuda")
    val.shortcut(paths, lengths, torch.zeros((0, 4, 2), device="cuda"))  # no steps
    assert torch.equal(paths, before) and lengths.tolist() == [6] * 4
    e = torch.zeros((0, 6, 7), device="cuda")
    val.shortcut(e, torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros((3, 0, 2), device="cuda"))
    with pytest.raises(vp.VPError):
        vp.vp_shortcut_paths(val.ctx, paths, lengths, torch.zeros((1, 4, 2), device="cuda"), -1.0)
    # a draw of (0, 1 - eps) proposes the first-to-last shortcut
    lengths.fill_(6)
    d = torch.tensor([[[0.0, 0.9999]]], device="cuda").repeat(1, 4, 1)
    val.shortcut(paths, lengths, d)
    cls, _ = oracle.Oracle(w.robot, w.env).classify_edges(before[:, 0].cpu().numpy(), before[:, 5].cpu().numpy(),
                                                          None, float(w.res))
    for p in range(4):
        if cls[p] != 2:
            assert lengths[p].item() == (2 if cls[p] == 0 else 6)
    val.close()
