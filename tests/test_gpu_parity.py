"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (from the method's numerics): sphere centres within 1e-5 m; state and
edge verdicts bit-exact wherever the oracle's clearance is outside the
1e-4 m band (band states / edges are counted, not compared); state counts
and every integer output bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import vpgen

pytestmark = pytest.mark.gpu

CENTRE_TOL = 1e-5
BAND = oracle.BAND


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    return Validator, vp


_cache = {}


def _setup(vpmod, name, n_edges):
    key = (name, n_edges)
    if key not in _cache:
        Validator, _ = vpmod
        w = vpgen.workload(name, n_edges=n_edges)
        _cache[key] = (w, Validator(w.robot, w.env), oracle.Oracle(w.robot, w.env))
    return _cache[key]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name", [vpgen.ARM7_SPHERES16, vpgen.TORSO8_OBB60_CAP20, vpgen.DUAL14_SHELVES])
def test_fk_centres(vpmod, name):
    w, val, o = _setup(vpmod, name, 64)
    q = vpgen.uniform_configs(w.robot, 4099, seed=31)  # ragged: not a multiple of the block
    got = val.fk_spheres(_cuda(q)).cpu().numpy()
    want = o.fk(q.astype(np.float64))
    err = np.abs(got - want).max()
    assert err <= CENTRE_TOL, err


def test_fk_general_tree_and_axes(vpmod):
    """A branching tree with general origin rotations and axes exercises the
    frame stash and the Rodrigues path."""
    from robots_small import EMPTY_ENV, random_chain
    Validator, _ = vpmod
    rng = np.random.default_rng(5)
    r = random_chain(rng, D=9, n_spheres=40)
    r.joint_parent = np.array([-1, 0, 1, 2, 1, 4, -1, 6, 3], dtype=np.int32)
    val = Validator(r, EMPTY_ENV)
    q = rng.uniform(-2, 2, size=(1000, 9)).astype(np.float32)
    got = val.fk_spheres(_cuda(q)).cpu().numpy()
    want = oracle.Oracle(r, EMPTY_ENV).fk(q.astype(np.float64))
    assert np.abs(got - want).max() <= CENTRE_TOL


def test_edge_counts_bit_exact(vpmod):
    w, val, o = _setup(vpmod, vpgen.ARM7_SPHERES16, 4096)
    got = val.edge_counts(_cuda(w.q0), _cuda(w.q1), w.res).cpu().numpy()
    assert np.array_equal(got, o.edge_count(w.q0, w.q1, w.res))
    # hand cases incl. the float32 decision, non-finite and over-long edges
    q0 = np.zeros((6, 7), np.float32)
    q1 = np.zeros((6, 7), np.float32)
    q0[1, 0], q1[1, 0] = np.float32(-1e-8), 1.0
    q1[2, 3] = np.nextafter(np.float32(1 / 32), np.float32(1))
    q0[3, 2] = np.nan
    q1[4, 6] = np.inf
    q1[5, 1] = 1e7
    got = val.edge_counts(_cuda(q0), _cuda(q1), w.res).cpu().numpy()
    assert list(got) == [2, 33, 3, -1, -1, -1]
    assert np.array_equal(got, o.edge_count(q0, q1, w.res))
    # the quotient is a float32 division: 0.3f / 0.1f rounds to 3.0f, so k = 4
    # (exact division would give 5)
    q1d = np.zeros((1, 7), np.float32)
    q1d[0, 0] = np.float32(0.3)
    got = val.edge_counts(_cuda(np.zeros((1, 7), np.float32)), _cuda(q1d), 0.1).cpu().numpy()
    assert list(got) == [4]


def _compare_states(val, o, q):
    got = val.validate_states(_cuda(q)).cpu().numpy()
    K = o.clearance(q.astype(np.float64))
    pinned = np.abs(K) > BAND
    bad = np.nonzero(got[pinned] != (K[pinned] >= 0))[0]
    return got, K, pinned, bad


@pytest.mark.parametrize("name", list(vpgen.NAMES))
def test_state_verdicts(vpmod, name):
    w, val, o = _setup(vpmod, name, 64)
    big = name == vpgen.DUAL14_MIXED1000
    q = vpgen.uniform_configs(w.robot, 1001 if big else 3001, seed=41 + vpgen.NAMES.index(name))
    got, K, pinned, bad = _compare_states(val, o, q)
    assert bad.size == 0, f"{bad.size} pinned states disagree"
    assert pinned.mean() > 0.99
    assert 0 < got.mean() < 1 or big


@pytest.mark.parametrize("name", [vpgen.TORSO8_OBB60_CAP20, vpgen.DUAL14_SHELVES])
def test_state_verdicts_wrapped_angles(vpmod, name):
    """The checks reduce each revolute angle to [-pi, pi] before the fast
    sine and cosine: the same configurations turned by whole turns (up to
    three either way, per joint) keep every pinned verdict of the oracle,
    which takes sin and cos of the unreduced angle in FP64."""
    w, val, o = _setup(vpmod, name, 64)
    q = vpgen.uniform_configs(w.robot, 3001, seed=47 + vpgen.NAMES.index(name))
    turns = np.random.default_rng(48).integers(-3, 4, size=q.shape)
    turns[:, w.robot.joint_type == vpgen.PRISMATIC] = 0
    qw = (q.astype(np.float64) + 2.0 * np.pi * turns).astype(np.float32)
    assert np.abs(qw).max() > 6 * np.pi
    got, K, pinned, bad = _compare_states(val, o, qw)
    assert bad.size == 0, f"{bad.size} pinned states disagree"
    assert pinned.mean() > 0.99
    assert 0 < got.mean() < 1


def _compare_edges(w, val, o, idx, mode, n_edges=None):
    from paper_2309_14545_gb300 import vp
    q0, q1 = _cuda(w.q0), _cuda(w.q1)
    counts = None if w.counts is None else _cuda(w.counts)
    got = val.validate_edges(q0, q1, counts, float(w.res), mode=mode).cpu().numpy()
    st, bits = val.sync_status()
    assert st == vp.VP_OK, (st, bits)
    c = None if w.counts is None else w.counts[idx]
    cls, nb = o.classify_edges(w.q0[idx], w.q1[idx], c, w.res)
    pinned = cls != 2
    bad = np.nonzero(got[idx][pinned] != (cls[pinned] == 0))[0]
    return got, cls, bad


def test_edges_arm7_every_edge(vpmod):
    """The 7-DoF arm workload at full size (10,000 edges): every pinned edge
    matches."""
    from paper_2309_14545_gb300 import vp
    w, val, o = _setup(vpmod, vpgen.ARM7_SPHERES16, None)
    idx = np.arange(w.q0.shape[0])
    got, cls, bad = _compare_edges(w, val, o, idx, vp.VP_MODE_PLAIN)
    assert bad.size == 0, f"{bad.size} pinned edges disagree"
    assert (cls == 2).mean() < 0.01
    assert 0.2 < got.mean() < 0.9


# Oracle subsets of the full-size workloads: 65,536 edges of the torso arm,
# the shelves and the 1,000-primitive scene (and of the mostly valid shelves
# variant); smaller ones where collision-free 512-state edges against 1,000
# primitives make the FP64 sweep long.
FULL_SIZE_SUBSETS = [(vpgen.TORSO8_OBB60_CAP20, 65536), (vpgen.DUAL14_SHELVES, 65536),
                     (vpgen.DUAL14_MIXED1000, 65536), (vpgen.DUAL14_SHELVES_MID, 65536),
                     (vpgen.DUAL14_MIXED1000_MID, 8192), (vpgen.DUAL14_SHELVES_FAR, 16384),
                     (vpgen.DUAL14_MIXED1000_FAR, 8192)]


@pytest.mark.parametrize("name,n_sample", FULL_SIZE_SUBSETS)
def test_edges_full_size_oracle_subset(vpmod, name, n_sample):
    """Full-size workloads in the benchmark's launch configuration (batched,
    autotuned on the whole batch; and one plain launch), checked on a seeded
    subset of edges the oracle classifies one by one: every pinned edge
    matches in both modes.  Band edges are counted and printed."""
    from paper_2309_14545_gb300 import vp
    w, val, o = _setup(vpmod, name, None)
    idx = np.sort(np.random.default_rng(n_sample + vpgen.NAMES.index(name)).choice(
        w.q0.shape[0], n_sample, replace=False))
    q0, q1 = _cuda(w.q0), _cuda(w.q1)
    counts = None if w.counts is None else _cuda(w.counts)
    val.autotune(q0, q1, counts, float(w.res))
    c = None if w.counts is None else w.counts[idx]
    cls, nb = o.classify_edges(w.q0[idx], w.q1[idx], c, w.res)
    pinned = cls != 2
    for mode in (vp.VP_MODE_BATCHED, vp.VP_MODE_PLAIN):
        got = val.validate_edges(q0, q1, counts, float(w.res), mode=mode).cpu().numpy()
        st, bits = val.sync_status()
        assert st == vp.VP_OK, (st, bits)
        bad = np.nonzero(got[idx][pinned] != (cls[pinned] == 0))[0]
        assert bad.size == 0, f"{name} mode {mode}: {bad.size} pinned edges disagree"
    print(f"{name}: {n_sample} oracle edges, {int((cls == 0).sum())} pinned free, {int((cls == 1).sum())} "
          f"pinned collide, {int((cls == 2).sum())} band edges, {int(nb.sum())} band states")
    assert (cls == 2).mean() < 0.01
    if name in (vpgen.DUAL14_SHELVES_MID, vpgen.DUAL14_MIXED1000_MID):
        assert (cls == 0).mean() >= 0.05  # mostly valid on purpose: full rakes are checked


def test_edge_edge_cases(vpmod):
    """Empty input, a single edge, two-state and constant edges, explicit
    maximum counts, non-finite endpoints and a count < 2 (reported through
    the device status word, edge invalid)."""
    from paper_2309_14545_gb300 import vp
    w, val, o = _setup(vpmod, vpgen.ARM7_SPHERES16, 2000)
    empty = torch.zeros((0, 7), dtype=torch.float32, device="cuda")
    out = val.validate_edges(empty, empty, None, float(w.res))
    assert out.numel() == 0
    n = 37  # ragged
    q0 = w.q0[:n].copy()
    q1 = w.q1[:n].copy()
    counts = np.full(n, 2, np.int32)
    counts[5:10] = 512
    q1[10:15] = q0[10:15]           # constant edges
    q0[15, 3] = np.nan              # non-finite endpoint
    q1[16, 0] = np.inf
    got = val.validate_edges(_cuda(q0), _cuda(q1), _cuda(counts), float(w.res)).cpu().numpy()
    st, bits = val.sync_status()
    assert st == vp.VP_OK
    cls, _ = o.classify_edges(q0, q1, counts, w.res)
    pinned = cls != 2
    assert np.array_equal(got[pinned], (cls[pinned] == 0).astype(np.uint8))
    assert got[15] == 0 and got[16] == 0
    counts[3] = 1
    got = val.validate_edges(_cuda(q0), _cuda(q1), _cuda(counts), float(w.res)).cpu().numpy()
    st, bits = val.sync_status()
    assert st == vp.VP_ERR_DEVICE and bits & vp.VP_DEVERR_COUNT
    assert got[3] == 0
    assert val.sync_status()[0] == vp.VP_OK  # cleared


def test_explicit_count_bound(vpmod):
    """An explicit count past the longest edge a resolution may give
    (VP_MAX_STEPS + 1 states) is refused on the device in every mode: the
    edge is invalid and the status word carries VP_DEVERR_LENGTH.  The
    largest accepted count is checked like any other.  Constant edges at a
    colliding configuration keep each accepted edge short to decide."""
    from paper_2309_14545_gb300 import vp
    w, val, o = _setup(vpmod, vpgen.ARM7_SPHERES16, 2000)
    K = o.clearance(w.q0.astype(np.float64))
    q_col = w.q0[np.nonzero(K < -0.01)[0][0]]
    q = _cuda(np.repeat(q_col[None], 4, axis=0))
    lim = vp.VP_MAX_STEPS + 1
    counts = np.array([lim, lim + 1, 2 ** 31 - 1, 2], np.int32)
    assert list(o.validate_edges(np.repeat(q_col[None], 4, 0), np.repeat(q_col[None], 4, 0), counts)) == [0] * 4
    for mode in (vp.VP_MODE_PLAIN, vp.VP_MODE_BATCHED):
        got = val.validate_edges(q, q, _cuda(counts), float(w.res), mode=mode).cpu().numpy()
        st, bits = val.sync_status()
        assert list(got) == [0, 0, 0, 0], mode
        assert st == vp.VP_ERR_DEVICE and bits == vp.VP_DEVERR_LENGTH, (mode, st, bits)
        got = val.validate_edges(q[:1], q[:1], _cuda(counts[:1]), float(w.res), mode=mode).cpu().numpy()
        assert list(got) == [0] and val.sync_status()[0] == vp.VP_OK, mode


def test_per_edge_launches_match_plain(vpmod):
    from paper_2309_14545_gb300 import vp
    w, val, o = _setup(vpmod, vpgen.DUAL14_SHELVES, 300)
    q0, q1, c = _cuda(w.q0), _cuda(w.q1), _cuda(w.counts)
    a = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PLAIN).cpu().numpy()
    b = val.validate_edges(q0, q1, c, float(w.res), mode=vp.VP_MODE_PER_EDGE).cpu().numpy()
    assert np.array_equal(a, b)


def test_work_counters(vpmod):
    from paper_2309_14545_gb300 import vp
    w, val, o = _setup(vpmod, vpgen.TORSO8_OBB60_CAP20, 4096)
    q0, q1 = _cuda(w.q0), _cuda(w.q1)
    a = val.validate_edges(q0, q1, None, float(w.res)).cpu().numpy()
    b, work = val.validate_edges_work(q0, q1, None, float(w.res))
    work = work.cpu().numpy()
    assert np.array_equal(a, b.cpu().numpy())
    assert work[vp.VP_WORK_EDGES_DONE] == 4096
    assert work[vp.VP_WORK_STATES] >= 4096
    # every posed state runs the coarse test of each sphere-carrying link
    # against every primitive until it stops
    assert work[vp.VP_WORK_COARSE_CUBOID] > 0 and work[vp.VP_WORK_COARSE_SPHERE] == 0


def test_argument_errors(vpmod):
    Validator, vp = vpmod
    w, val, o = _setup(vpmod, vpgen.ARM7_SPHERES16, 64)
    bad = vpgen.arm7(0, 40)
    bad.joint_parent = np.array([-1, 0, 5, 2, 3, 4, 5], dtype=np.int32)  # parent after child
    with pytest.raises(vp.VPError) as e:
        vp.vp_load_robot(val.ctx, bad)
    assert e.value.status == vp.VP_ERR_ARG
    big = vpgen.Env(np.zeros((20000, 4)) + [0, 0, 0, 0.1], np.zeros((0, 7)), np.zeros((0, 15)))
    with pytest.raises(vp.VPError) as e:
        vp.vp_load_env(val.ctx, big)
    assert e.value.status == vp.VP_ERR_CAPACITY
    q = torch.zeros((4, 7), device="cuda")
    with pytest.raises(vp.VPError) as e:
        val.validate_edges(q, q, None, 0.0)
    assert e.value.status == vp.VP_ERR_ARG


@pytest.mark.parametrize("D,parents", [
    (9, [-1, 0, 1, 2, 1, 4, -1, 6, 3]),                                     # tree, 10 links
    (16, [-1, 0, 1, 2, 3, 4, 2, 6, 7, -1, 9, 10, 11, 10, 13, 14]),        # 17 links
])
def test_tree_robot_general_axes_states_and_edges(vpmod, D, parents):
    """Branching robots with general axes and origin rotations, prismatic
    joints and self pairs across branches, against the oracle: the pose
    pass restores branch-point frames, the general joint code, and the
    17-link kernel instance."""
    from robots_small import random_chain
    Validator, vp = vpmod
    rng = np.random.default_rng(100 + D)
    r = random_chain(rng, D=D, n_spheres=60)
    r.joint_parent = np.array(parents, dtype=np.int32)
    links = r.sphere_link
    cand = [(a, b) for a in range(60) for b in range(a + 1, 60) if abs(int(links[a]) - int(links[b])) >= 2]
    r.self_pairs = np.array([cand[i] for i in rng.choice(len(cand), 80, replace=False)], dtype=np.int32)
    env = vpgen.Env(np.array([[0.3, 0.2, 0.1, 0.15], [-0.3, 0.1, 0.2, 0.1]]),
                    np.array([[0.0, -0.4, 0.0, 0.3, -0.2, 0.3, 0.06]]),
                    np.array([np.concatenate([[0.1, 0.4, -0.2], np.eye(3).ravel(), [0.15, 0.1, 0.1]])]))
    val = Validator(r, env)
    o = oracle.Oracle(r, env)
    q = rng.uniform(-1.5, 1.5, size=(2000, D)).astype(np.float32)
    got, K, pinned, bad = _compare_states(val, o, q)
    assert bad.size == 0 and 0.05 < got.mean() < 0.95
    q0, q1 = q[:600], rng.uniform(-1.5, 1.5, size=(600, D)).astype(np.float32)
    counts = rng.integers(2, 40, size=600).astype(np.int32)
    for mode in (vp.VP_MODE_PLAIN, vp.VP_MODE_BATCHED):
        v = val.validate_edges(_cuda(q0), _cuda(q1), _cuda(counts), 1 / 32, mode=mode).cpu().numpy()
        cls, _ = o.classify_edges(q0, q1, counts, np.float32(1 / 32))
        pinned = cls != 2
        assert np.array_equal(v[pinned], (cls[pinned] == 0).astype(np.uint8)), mode
