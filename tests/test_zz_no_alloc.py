"""The allocation-free edge validation entry point.

vp_validate_edges_noalloc serves callers that must not allocate device
memory while they run (a planner inside a robot's real-time control loop,
a process whose device memory is fixed at start-up): it needs no context
and keeps its scratch -- the packed environment and the status word -- in
a static device array of the library.  Through the C ABI it must give the
same verdicts as vp_validate_edges (plain mode) -- exactly, as every
integer output here -- on consecutive calls that reuse the shared array
with different environments, and it must reject an environment larger
than the array before running anything.

This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import vpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    return Validator, vp


def _reference(Validator, w):
    val = Validator(w.robot, w.env)
    q0, q1 = torch.from_numpy(w.q0).cuda(), torch.from_numpy(w.q1).cuda()
    c = None if w.counts is None else torch.from_numpy(w.counts).cuda()
    out = val.validate_edges(q0, q1, c, float(w.res)).cpu().numpy()
    val.close()
    return q0, q1, c, out


def test_noalloc_matches_plain_on_consecutive_calls(vpmod):
    Validator, vp = vpmod
    cases = [vpgen.workload(vpgen.TORSO8_OBB60_CAP20, n_edges=20_003),
             vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=10_000),
             vpgen.workload(vpgen.DUAL14_SHELVES, n_edges=5_001)]
    for w in cases + cases[:1]:  # the last call follows a different environment
        q0, q1, c, want = _reference(Validator, w)
        got = torch.full((w.q0.shape[0],), 7, dtype=torch.uint8, device="cuda")
        vp.vp_validate_edges_noalloc(w.robot, w.env, q0, q1, c, float(w.res), got)
        assert np.array_equal(got.cpu().numpy(), want), w.name
        assert 0 < want.mean() < 1 or w.name == vpgen.DUAL14_SHELVES


def test_noalloc_rejects_an_environment_beyond_the_scratch(vpmod):
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=64)
    n = vp.VP_NOALLOC_MAX_ENV_BYTES // 96 + 1  # cuboids pack to 96 bytes each
    big = vpgen.Env(np.zeros((0, 4)), np.zeros((0, 7)),
                    np.tile(np.concatenate([[5.0, 5, 5], np.eye(3).ravel(), [0.1, 0.1, 0.1]]), (n, 1)))
    q0, q1 = torch.from_numpy(w.q0).cuda(), torch.from_numpy(w.q1).cuda()
    got = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(vp.VPError) as e:
        vp.vp_validate_edges_noalloc(w.robot, big, q0, q1, None, float(w.res), got)
    assert e.value.status == vp.VP_ERR_CAPACITY
    assert "static scratch" in str(e.value)
