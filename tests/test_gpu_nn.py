"""Batched l2 nearest neighbours (vp_nearest) against the FP64 oracle.

Where the oracle's best and second-best distances are apart by more than the
FP32 rounding of a distance (relative 1e-5), the index must be the oracle's;
inside that gap any index whose FP64 distance is within it is correct (the
FP32 order decides).  Distances match the FP64 distance of the returned
point to relative 1e-5."""
import numpy as np
import pytest
import torch

from oracle.nn import nearest

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    import vpgen
    return Validator(vpgen.robot_for(vpgen.ARM7_SPHERES16), vpgen.env_for(vpgen.ARM7_SPHERES16)), vp


def _check(p, q, idx, d2):
    want_i, want_d, second = nearest(p, q)
    got_d64 = ((q - p[idx]) ** 2).sum(axis=1)
    scale = TOL * (1.0 + want_d)
    unique = second - want_d > scale
    assert np.array_equal(idx[unique], want_i[unique])
    assert np.all(got_d64 <= want_d + scale)  # elsewhere: a nearest point up to rounding
    np.testing.assert_allclose(d2, got_d64, rtol=TOL, atol=1e-7)
    return unique.mean()


@pytest.mark.parametrize("M,N,D", [(1, 5, 3), (1000, 1, 7), (3, 1000, 1), (20_000, 300, 14), (5_000, 17, 16),
                                   (100_000, 4096, 7), (777, 2049, 5), (130, 9, 2)])
def test_nearest_matches_oracle(vpmod, M, N, D):
    val, vp = vpmod
    rng = np.random.default_rng(M * 31 + N + D)
    p = rng.uniform(-2.8, 2.8, size=(M, D)).astype(np.float32)
    q = rng.uniform(-2.8, 2.8, size=(N, D)).astype(np.float32)
    idx, d2 = val.nearest(torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda())
    frac = _check(p.astype(np.float64), q.astype(np.float64), idx.cpu().numpy(), d2.cpu().numpy().astype(np.float64))
    assert frac > 0.9


def test_full_size_sampled(vpmod):
    """The benchmark's case (1,048,576 points, 4,096 queries, D = 7), checked
    on a seeded sample of 256 queries."""
    val, vp = vpmod
    rng = np.random.default_rng(77)
    p = rng.uniform(-2.8, 2.8, size=(1 << 20, 7)).astype(np.float32)
    q = rng.uniform(-2.8, 2.8, size=(4096, 7)).astype(np.float32)
    idx, d2 = val.nearest(torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda())
    s = np.sort(rng.choice(4096, 256, replace=False))
    _check(p.astype(np.float64), q[s].astype(np.float64), idx.cpu().numpy()[s], d2.cpu().numpy()[s].astype(np.float64))


def test_ties_take_the_lowest_index_and_nonfinite_points_never_win(vpmod):
    val, vp = vpmod
    p = np.array([[0, 0, 0], [2, 0, 0], [0, 2, 0], [2, 0, 0], [np.nan, 0, 0], [1, 0, 0]], np.float32)
    p = np.concatenate([p, np.full((3000, 3), 50.0, np.float32)])  # several tiles
    p[2500] = [1, 0, 0]  # a later duplicate of point 5
    q = np.array([[1, 1, 0], [2.25, 0, 0], [1, 0, 0], [0.75, 0, 0]], np.float32)
    idx, d2 = val.nearest(torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda())
    # query 0: point 5 at 1 (points 0-3 at 2); query 1: points 1 and 3 tie at
    # 1/16, the lower wins; query 2: points 5 and 2500 tie at 0 (different
    # tiles and blocks); query 3: point 5 at 1/16.  The NaN point never wins.
    assert idx.cpu().tolist() == [5, 1, 5, 5]
    np.testing.assert_array_equal(d2.cpu().numpy(), [1.0, 0.0625, 0.0, 0.0625])


def test_edge_cases(vpmod):
    val, vp = vpmod
    p = torch.rand(10, 4, device="cuda")
    idx, d2 = val.nearest(p, torch.empty(0, 4, device="cuda"))
    assert idx.numel() == 0
    with pytest.raises(vp.VPError):
        val.nearest(torch.empty(0, 4, device="cuda"), p)
    with pytest.raises(vp.VPError):
        val.nearest(torch.rand(5, 17, device="cuda"), torch.rand(3, 17, device="cuda"))
    allnan = torch.full((4, 2), float("nan"), device="cuda")
    idx, _ = val.nearest(allnan, torch.zeros(2, 2, device="cuda"))
    assert idx.cpu().tolist() == [-1, -1]
