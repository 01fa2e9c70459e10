"""Batched mode (length-bucketed persistent kernel replayed from a CUDA
graph, tiling from the autotuner) against the plain kernel and the oracle.

Verdicts of the two modes must agree bit for bit on every edge (same
arithmetic, only the lane assignment differs), and pinned edges must agree
with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import vpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    return Validator, vp


def _cuda(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same_outside_band(w, got, want, idx=None):
    """Verdicts of two check orders: both families pose the links with the
    same arithmetic but rebuild link frames along different float paths, so
    they may differ only where the oracle puts the edge in the boundary band
    (some state within 1e-4 m of contact)."""
    diff = np.nonzero(got != want)[0]
    if diff.size == 0:
        return 0
    o = oracle.Oracle(w.robot, w.env)
    e = diff if idx is None else idx[diff]
    c = None if w.counts is None else w.counts[e]
    cls, _ = o.classify_edges(w.q0[e], w.q1[e], c, w.res)
    assert np.all(cls == 2), f"{int((cls != 2).sum())} edges outside the band differ"
    return int(diff.size)


def _same_states_outside_band(w, q, got, want):
    diff = np.nonzero(got != want)[0]
    if diff.size == 0:
        return 0
    K = oracle.Oracle(w.robot, w.env).clearance(q[diff].astype(np.float64))
    assert np.all(np.abs(K) <= oracle.BAND), f"{int((np.abs(K) > oracle.BAND).sum())} states outside the band differ"
    return int(diff.size)


def _both(val, vp, w, tune):
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    if tune:  # the tuned check order is the plain kernel's too
        val.autotune(q0, q1, c, float(w.res))
    plain = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
    out = torch.full((w.q0.shape[0],), 9, dtype=torch.uint8, device="cuda")
    val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED, out=out)
    first = out.cpu().numpy()
    out.fill_(9)
    val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED, out=out)  # graph replay
    assert val.sync_status()[0] == vp.VP_OK
    return plain, first, out.cpu().numpy()


@pytest.mark.parametrize("name,n,tune", [(vpgen.ARM7_SPHERES16, None, False), (vpgen.ARM7_SPHERES16, None, True),
                                         (vpgen.DUAL14_SHELVES, None, True), (vpgen.DUAL14_MIXED1000, 300_000, True),
                                         (vpgen.TORSO8_OBB60_CAP20, 200_000, True)])
def test_batched_equals_plain(vpmod, name, n, tune):
    Validator, vp = vpmod
    w = vpgen.workload(name, n_edges=n)
    val = Validator(w.robot, w.env)
    plain, b1, b2 = _both(val, vp, w, tune)
    assert np.array_equal(plain, b1) and np.array_equal(plain, b2)
    val.close()


def test_batched_mixed_lengths_against_oracle(vpmod):
    """Every length bucket (2 .. 1000 states) in one batch, ragged size,
    explicit counts; pinned edges match the oracle."""
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=3001)
    rng = np.random.default_rng(9)
    counts = rng.choice([2, 3, 4, 5, 8, 9, 16, 17, 31, 32, 33, 64, 65, 200, 256, 257, 512, 700, 1000],
                        size=3001).astype(np.int32)
    val = Validator(w.robot, w.env)
    q0, q1 = _cuda(w.q0), _cuda(w.q1)
    val.autotune(q0, q1, _cuda(counts), float(w.res))
    got = val.validate_edges(q0, q1, _cuda(counts), float(w.res), mode=vp.VP_MODE_BATCHED).cpu().numpy()
    plain = val.validate_edges(q0, q1, _cuda(counts), float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
    assert np.array_equal(got, plain)
    cls, _ = oracle.Oracle(w.robot, w.env).classify_edges(w.q0, w.q1, counts, w.res)
    pinned = cls != 2
    assert np.array_equal(got[pinned], (cls[pinned] == 0).astype(np.uint8))
    assert 0 < got.mean() < 1


def test_batched_edge_cases(vpmod):
    """Bad counts are answered in the bucketing pass (invalid + device
    status); non-finite endpoints make an edge invalid -- in the edge kernel
    with explicit counts (in every length bucket, so at every lane-group
    size), in the bucketing pass without; tiny and empty batches; new
    buffers after a graph was built."""
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.DUAL14_SHELVES, n_edges=70)
    val = Validator(w.robot, w.env)
    counts = w.counts.copy()
    counts[3] = 0
    q0, q1 = w.q0.copy(), w.q1.copy()
    q0[5, 2] = np.nan
    q1[6, 13] = np.inf
    q0[7, 0] = -np.inf
    bad = [5, 6, 7]
    for i, k in zip(range(8, 17), (2, 5, 9, 17, 33, 65, 129, 257, 512)):  # one per bucket
        counts[i] = k
        q1[i, i % 14] = np.nan
        bad.append(i)
    got = val.validate_edges(_cuda(q0), _cuda(q1), _cuda(counts), float(w.res), mode=vp.VP_MODE_BATCHED)
    st, bits = val.sync_status()
    assert st == vp.VP_ERR_DEVICE and bits == vp.VP_DEVERR_COUNT
    got = got.cpu().numpy()
    assert got[3] == 0 and np.all(got[bad] == 0)
    plain = val.validate_edges(_cuda(q0), _cuda(q1), _cuda(counts), float(w.res)).cpu().numpy()
    val.sync_status()
    assert np.array_equal(got, plain)
    for lanes in ([4] * 9, [32] * 9):
        val.set_tiling(lanes)
        again = val.validate_edges(_cuda(q0), _cuda(q1), _cuda(counts), float(w.res), mode=vp.VP_MODE_BATCHED)
        val.sync_status()
        assert np.array_equal(again.cpu().numpy(), plain), lanes
    got = val.validate_edges(_cuda(q0), _cuda(q1), None, float(w.res), mode=vp.VP_MODE_BATCHED).cpu().numpy()
    assert val.sync_status()[0] == vp.VP_OK
    assert np.all(got[bad] == 0)
    assert np.array_equal(got, val.validate_edges(_cuda(q0), _cuda(q1), None, float(w.res)).cpu().numpy())
    for n in (1, 2, 33):
        a = val.validate_edges(_cuda(w.q0[:n]), _cuda(w.q1[:n]), _cuda(w.counts[:n]), float(w.res),
                               mode=vp.VP_MODE_BATCHED).cpu().numpy()
        b = val.validate_edges(_cuda(w.q0[:n]), _cuda(w.q1[:n]), _cuda(w.counts[:n]), float(w.res)).cpu().numpy()
        assert np.array_equal(a, b)
    e = torch.zeros((0, 14), device="cuda")
    assert val.validate_edges(e, e, None, float(w.res), mode=vp.VP_MODE_BATCHED).numel() == 0
    assert val.sync_status()[0] == vp.VP_OK


def test_batched_work_counters(vpmod):
    """The counting variant of the batched kernel gives the same verdicts and
    finishes every edge exactly once."""
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.DUAL14_SHELVES, n_edges=20_000)
    val = Validator(w.robot, w.env)
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    plain = val.validate_edges(q0, q1, c, float(w.res)).cpu().numpy()
    got, work = val.validate_edges_work(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED)
    work = work.cpu().numpy()
    assert np.array_equal(got.cpu().numpy(), plain)
    assert work[vp.VP_WORK_EDGES_DONE] == 20_000
    assert work[vp.VP_WORK_STATES] >= 20_000 * 2 * 0  # at least one state per edge that is posed
    assert work[vp.VP_WORK_STATES] <= int(w.counts.astype(np.int64).sum())
    # lane slots: every lane of a running warp, so whole warps, and at least the live work
    coarse = work[[vp.VP_WORK_COARSE_SPHERE, vp.VP_WORK_COARSE_CAPSULE, vp.VP_WORK_COARSE_CUBOID]].sum()
    fine = work[[vp.VP_WORK_FINE_SPHERE, vp.VP_WORK_FINE_CAPSULE, vp.VP_WORK_FINE_CUBOID]].sum()
    for slot, live in ((vp.VP_WORK_LANE_STATES, work[vp.VP_WORK_STATES]), (vp.VP_WORK_LANE_COARSE, coarse),
                       (vp.VP_WORK_LANE_FINE, fine), (vp.VP_WORK_LANE_PAIR_FINE, work[vp.VP_WORK_PAIR_FINE])):
        assert work[slot] % 32 == 0 and work[slot] >= live > 0
    # lanes whose own coarse test hit are a subset of the live lanes
    assert 0 < work[vp.VP_WORK_FINE_OWN] <= fine
    assert 0 < work[vp.VP_WORK_PAIR_FINE_OWN] <= work[vp.VP_WORK_PAIR_FINE]


@pytest.mark.parametrize("name,n", [(vpgen.TORSO8_OBB60_CAP20, 60_000), (vpgen.DUAL14_MIXED1000, 60_000),
                                    (vpgen.ARM7_SPHERES16, 30_000)])
def test_second_phase_matches_plain(vpmod, name, n):
    """Edges handed to the second launch (after 1, 2 or 4 screening rounds,
    or none) get the verdicts of the plain kernel, at several tilings, in the
    default order and in the two-pass order (whose first pass hands edges to
    a second screening launch as well)."""
    Validator, vp = vpmod
    w = vpgen.workload(name, n_edges=n)
    val = Validator(w.robot, w.env)
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    want = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
    assert 0 < want.mean() < 1
    for order in (0, vp.VP_ORDER_FREQUENT_TWO_PASS):
        val.set_check_order(order)
        want_o = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
        for rounds in (1, 2, 4, 0):
            val.set_screen_rounds(rounds)
            assert val.screen_rounds() == rounds
            for lanes in ([4] * 9, [32] * 9, [4, 8, 16, 8, 4, 16, 8, 32, 16]):
                val.set_tiling(lanes)
                out = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
                val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED, out=out)
                assert np.array_equal(out.cpu().numpy(), want_o), (order, rounds, lanes)
    val.set_check_order(0)
    # the other check orders (primitives first; checks interleaved with
    # posing, either way round; frequent link pairs first with links posed
    # on demand): within one order every mode and setting gives the same
    # verdicts bit for bit; across orders they agree outside the band
    states = q0[: min(n, 20000)]
    want_s = val.validate_states(states).cpu().numpy()
    qs = w.q0[: min(n, 20000)]
    for order in (1, 2, 3, 4, 5):
        val.set_check_order(order)
        assert val.check_order() == order
        ref = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
        ndiff = _same_outside_band(w, ref, want)
        got = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED).cpu().numpy()
        assert np.array_equal(got, ref), order
        got, work = val.validate_edges_work(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED)
        assert np.array_equal(got.cpu().numpy(), ref), order
        assert int(work[vp.VP_WORK_EDGES_DONE]) == n
        nds = _same_states_outside_band(w, qs, val.validate_states(states).cpu().numpy(), want_s)
        print(f"{name} order {order}: {ndiff} band edges and {nds} band states differ from order 0")
    val.set_check_order(0)
    assert val.sync_status()[0] == vp.VP_OK
    with pytest.raises(vp.VPError):
        val.set_screen_rounds(-1)
    for bad in (-1, 6):
        with pytest.raises(vp.VPError):
            val.set_check_order(bad)
    # the frequent-first order after the tuner has counted the groups
    val.autotune(q0, q1, c, float(w.res))
    for order in (4, 5):
        val.set_check_order(order)
        ref = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
        _same_outside_band(w, ref, want)
        got = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED).cpu().numpy()
        assert np.array_equal(got, ref), ("tuned", order)
        _same_states_outside_band(w, qs, val.validate_states(states).cpu().numpy(), want_s)
    val.close()


def test_measured_fp32_peak(vpmod):
    """The FMA-chain measurement gives a plausible device rate and rejects
    bad arguments."""
    Validator, vp = vpmod
    t = vp.vp_measure_fp32_peak(0, 0.2)
    props = torch.cuda.get_device_properties(0)
    derived_at_3ghz = 2 * 128 * props.multi_processor_count * 3.0e9 / 1e12
    assert 0.2 * derived_at_3ghz / 3 < t < derived_at_3ghz
    with pytest.raises(vp.VPError):
        vp.vp_measure_fp32_peak(0, 0.0)


def test_tiling_defaults_then_tuned(vpmod):
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.DUAL14_SHELVES, n_edges=100_000)
    val = Validator(w.robot, w.env)
    assert val.tiling() == [4, 8, 16, 32, 32, 32, 32, 32, 32]
    val.autotune(_cuda(w.q0), _cuda(w.q1), _cuda(w.counts), float(w.res))
    t = val.tiling()
    assert len(t) == 9 and set(t) <= {4, 8, 16, 32}
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    want = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
    for lanes in ([32] * 9, [4] * 9, [8, 16]):
        val.set_tiling(lanes)
        assert val.tiling()[:len(lanes)] == lanes
        got = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED).cpu().numpy()
        assert np.array_equal(got, want)
    for bad in ([3], [64], [4] * 10):
        with pytest.raises(vp.VPError):
            val.set_tiling(bad)
    assert val.tiling()[:2] == [8, 16]
    val.close()


def test_kernel_timing_hook(vpmod):
    """vp_kernel_time reports the validation kernel's own duration, for both
    modes (inside the replayed graph for batched)."""
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.DUAL14_SHELVES, n_edges=50_000)
    val = Validator(w.robot, w.env)
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    assert val.kernel_time(True) == -1.0
    for mode in (vp.VP_MODE_PLAIN, vp.VP_MODE_BATCHED, vp.VP_MODE_BATCHED):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        val.validate_edges(q0, q1, c, float(w.res), mode=mode)
        b.record()
        b.synchronize()
        k = val.kernel_time(True)
        assert 0.0 < k <= a.elapsed_time(b) * 1.05 + 0.01
    val.kernel_time(False)


def test_watchdog_reports_timeout_and_context_survives(vpmod):
    """A zero time budget makes the persistent kernel give up at once: the
    device status reports VP_ERR_TIMEOUT (no fault, no hang), and the same
    context then validates correctly with the budget restored."""
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.DUAL14_SHELVES, n_edges=4096)
    val = Validator(w.robot, w.env)
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    vp.vp_set_watchdog(val.ctx, 0.0)
    val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED)
    st, bits = val.sync_status()
    assert st == vp.VP_ERR_TIMEOUT and bits & vp.VP_DEVERR_TIMEOUT
    vp.vp_set_watchdog(val.ctx, 60.0)
    got = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED).cpu().numpy()
    assert val.sync_status()[0] == vp.VP_OK
    plain = val.validate_edges(q0, q1, c, float(w.res)).cpu().numpy()
    assert np.array_equal(got, plain)
    with pytest.raises(vp.VPError):
        vp.vp_set_watchdog(val.ctx, -1.0)


@pytest.mark.parametrize("case", ["no_self_pairs", "no_primitives"])
def test_two_pass_order_edge_cases(vpmod, case):
    """The two-pass order where its first pass decides nothing (a robot with
    no self pairs: every edge is deferred) and where the second has no
    primitives to check (an empty scene): batched verdicts equal the plain
    kernel's at several tilings and screening rounds, and pinned edges of a
    subset match the oracle."""
    import dataclasses
    from robots_small import EMPTY_ENV
    Validator, vp = vpmod
    w = vpgen.workload(vpgen.DUAL14_MIXED1000, n_edges=40_000)
    robot, env = w.robot, w.env
    if case == "no_self_pairs":
        robot = dataclasses.replace(robot, self_pairs=np.zeros((0, 2), dtype=np.int32))
    else:
        env = EMPTY_ENV
    val = Validator(robot, env)
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    val.autotune(q0, q1, c, float(w.res))
    val.set_check_order(vp.VP_ORDER_FREQUENT_TWO_PASS)
    want = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
    for rounds in (1, 0):
        val.set_screen_rounds(rounds)
        for lanes in ([4] * 9, [4, 8, 16, 32, 32, 32, 32, 32, 32]):
            val.set_tiling(lanes)
            got = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED).cpu().numpy()
            assert np.array_equal(got, want), (case, rounds, lanes)
    got, work = val.validate_edges_work(q0, q1, c, float(w.res), mode=vp.VP_MODE_BATCHED)
    assert np.array_equal(got.cpu().numpy(), want)
    assert int(work[vp.VP_WORK_EDGES_DONE]) == w.q0.shape[0]
    assert val.sync_status()[0] == vp.VP_OK
    idx = np.arange(0, w.q0.shape[0], 80)
    cls, _ = oracle.Oracle(robot, env).classify_edges(w.q0[idx], w.q1[idx], w.counts[idx], w.res)
    pinned = cls != 2
    assert np.array_equal(want[idx][pinned], (cls[pinned] == 0).astype(np.uint8))
    val.close()
