"""Batched RRT-Connect (vp_rrt_connect) against the oracle's RRT-Connect
run on the same samples.  The trees are shaped by FP32 decisions both sides
take with the same rounding, and by edge verdicts: wherever no edge verdict
(and neither endpoint) fell inside the clearance band, status, samples used,
tree sizes and the path must be identical; otherwise the GPU's path must
still be a valid path from start to goal."""
import numpy as np
import pytest
import torch

import oracle
import vpgen
from oracle.rrt import rrt_connect

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    return Validator, vp


def _problems(robot, B, T, seed):
    start, goal = vpgen.uniform_edges(robot, B, seed=seed)
    samples = np.stack([vpgen.uniform_configs(robot, T, seed=seed + 1000 + b) for b in range(B)])
    return start, goal, samples


@pytest.mark.parametrize("name,B,T,rng,cap", [(vpgen.ARM7_SPHERES16, 40, 300, 1.0, 512),
                                              (vpgen.TORSO8_OBB60_CAP20, 12, 150, 0.8, 256)])
def test_rrt_connect_matches_oracle(vpmod, name, B, T, rng, cap):
    Validator, vp = vpmod
    w = vpgen.workload(name, n_edges=8)
    start, goal, samples = _problems(w.robot, B, T, seed=61)
    val = Validator(w.robot, w.env)
    out = val.rrt_connect(torch.from_numpy(start).cuda(), torch.from_numpy(goal).cuda(),
                          torch.from_numpy(samples).cuda(), rng, float(w.res), cap)
    assert val.sync_status()[0] == vp.VP_OK
    got = {k: v.cpu().numpy() for k, v in out.items()}
    o = oracle.Oracle(w.robot, w.env)
    compared = solved = 0
    for b in range(B):
        st, it, path, band, sizes = rrt_connect(o, start[b], goal[b], samples[b], rng, float(w.res), cap)
        gp = got["path"][b, :got["path_len"][b]]
        if got["status"][b] == 1:
            solved += 1
            np.testing.assert_array_equal(gp[0], start[b])
            np.testing.assert_array_equal(gp[-1], goal[b])
            cls, _ = o.classify_edges(gp[:-1], gp[1:], None, float(w.res))
            assert np.all(cls != 1), b  # no pinned-colliding edge on a returned path
        if band:
            continue
        compared += 1
        assert got["status"][b] == st and got["iters"][b] == it, b
        assert tuple(got["tree_sizes"][b]) == sizes, b
        if st == 1:
            np.testing.assert_array_equal(gp, path)
        else:
            assert got["path_len"][b] == 0
    assert compared >= 0.7 * B and solved >= 1
    val.close()


@pytest.mark.parametrize("T", [300, 40])
def test_rrt_connect_second_phase_matches_oracle(vpmod, T):
    """Problems that outlast the first phase's 32 samples are resumed by a
    team of warps (T = 300: most are solved there; T = 40: some run out of
    samples there).  Endpoints are drawn where the oracle finds clearance
    above 1 mm, so every problem plans; outcomes must match the oracle's
    exactly wherever no edge verdict fell inside the band."""
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.TORSO8_OBB60_CAP20, n_edges=8)
    o = oracle.Oracle(w.robot, w.env)
    cand = vpgen.uniform_configs(w.robot, 1200, seed=71)
    free = cand[o.clearance(cand.astype(np.float64)) > 1e-3]
    B = 96
    start, goal = free[:B], free[B:2 * B]
    samples = np.stack([vpgen.uniform_configs(w.robot, T, seed=1071 + b) for b in range(B)])
    val = Validator(w.robot, w.env)
    out = val.rrt_connect(torch.from_numpy(start).cuda(), torch.from_numpy(goal).cuda(),
                          torch.from_numpy(samples).cuda(), 0.8, float(w.res), 512)
    assert val.sync_status()[0] == vp.VP_OK
    got = {k: v.cpu().numpy() for k, v in out.items()}
    compared = long_runs = 0
    for b in range(B):
        st, it, path, band, sizes = rrt_connect(o, start[b], goal[b], samples[b], 0.8, float(w.res), 512)
        if band:
            continue
        compared += 1
        long_runs += it > 32
        assert got["status"][b] == st and got["iters"][b] == it, b
        assert tuple(got["tree_sizes"][b]) == sizes, b
        if st == 1:
            np.testing.assert_array_equal(got["path"][b, :got["path_len"][b]], path)
        else:
            assert got["path_len"][b] == 0
    assert compared >= 0.8 * B and long_runs >= 5


def test_rrt_connect_edge_cases(vpmod):
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=8)
    val = Validator(w.robot, w.env)
    start, goal, samples = _problems(w.robot, 4, 5, seed=3)
    s, g, q = (torch.from_numpy(x).cuda() for x in (start, goal, samples))
    out = val.rrt_connect(s, g, q[:, :0].contiguous(), 1.0, float(w.res), 16)  # no samples
    st = out["status"].cpu().numpy()
    assert np.all((st == 0) | (st == -1)) and np.all(out["path_len"].cpu().numpy() == 0)
    out = val.rrt_connect(s, s.clone(), q, 1.0, float(w.res), 16)  # start == goal
    o = oracle.Oracle(w.robot, w.env)
    k = o.clearance(start.astype(np.float64))
    for b in range(4):
        if abs(k[b]) > 1e-4:
            assert out["status"][b].item() == (1 if k[b] > 0 else -1)
    with pytest.raises(vp.VPError):
        val.rrt_connect(s, g, q, -1.0, float(w.res), 16)
    with pytest.raises(vp.VPError):
        val.rrt_connect(s, g, q, 1.0, float(w.res), 1)
    val.close()
