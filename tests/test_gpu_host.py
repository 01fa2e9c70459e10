"""Edge validation from host memory (vp_validate_edges_host): the batch cut
into chunks whose copies overlap the work must give exactly the verdicts of
vp_validate_edges on the same arrays held on the device, in both modes, for
one chunk and several (with a ragged last one), with explicit counts and
without, from page-locked and from pageable memory, and again on a repeated
call (the batched mode replays one graph per chunk)."""
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


@pytest.mark.parametrize("name,n", [(vpgen.DUAL14_MIXED1000, 1_200_003), (vpgen.TORSO8_OBB60_CAP20, 1_100_001),
                                    (vpgen.TORSO8_OBB60_CAP20, 777),
                                    (vpgen.ARM7_SPHERES16, 1)])
def test_host_equals_device(vpmod, name, n):
    Validator, vp = vpmod
    w = vpgen.workload(name, n_edges=n)
    val = Validator(w.robot, w.env)
    q0, q1 = torch.from_numpy(w.q0), torch.from_numpy(w.q1)
    c = None if w.counts is None else torch.from_numpy(w.counts)
    d0, d1 = q0.cuda(), q1.cuda()
    dc = None if c is None else c.cuda()
    val.autotune(d0, d1, dc, float(w.res))
    p0, p1 = q0.pin_memory(), q1.pin_memory()
    pc = None if c is None else c.pin_memory()
    for mode in (vp.VP_MODE_PLAIN, vp.VP_MODE_BATCHED):
        want = val.validate_edges(d0, d1, dc, float(w.res), mode=mode).cpu().numpy()
        for rep in range(2):
            out = val.validate_edges_host(p0, p1, pc, float(w.res), mode=mode)
            torch.cuda.synchronize()
            assert np.array_equal(out.numpy(), want), (mode, rep)
        pageable = torch.full((n,), 9, dtype=torch.uint8)
        val.validate_edges_host(q0, q1, c, float(w.res), mode=mode, out=pageable)
        torch.cuda.synchronize()
        assert np.array_equal(pageable.numpy(), want), mode
    assert val.sync_status()[0] == vp.VP_OK
    val.close()


def test_host_counts_from_resolution_and_errors(vpmod):
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.DUAL14_SHELVES, n_edges=70_000)
    val = Validator(w.robot, w.env)
    q0, q1 = torch.from_numpy(w.q0).pin_memory(), torch.from_numpy(w.q1).pin_memory()
    want = val.validate_edges(q0.cuda(), q1.cuda(), None, float(w.res)).cpu().numpy()
    out = val.validate_edges_host(q0, q1, None, float(w.res))
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), want)
    with pytest.raises(vp.VPError):
        val.validate_edges_host(q0, q1, None, float(w.res), mode=vp.VP_MODE_PER_EDGE)
    with pytest.raises(TypeError):
        val.validate_edges_host(q0.cuda(), q1.cuda(), None, float(w.res))
    empty = torch.zeros((0, 14), dtype=torch.float32)
    assert val.validate_edges_host(empty, empty, None, float(w.res)).numel() == 0
    val.close()
