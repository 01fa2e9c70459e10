"""Penetration cost and its reverse-mode FK adjoint against the FP64 oracle.

Bars:
- cost within rtol 1e-4 (+1e-6 absolute);
- gradient, per sample, rel = max_j |g_gpu,j - g_ref,j| / max_j |g_ref,j|:
  rel <= 1e-3 on every sample whose root-sum-square penetration sqrt(cost)
  exceeds the 1e-4 m clearance band the verdicts use and whose oracle
  gradient is resolvable in float32: it moves by at most 1e-3 (relative)
  when q moves by 1e-6 rad (about eight float32 ulps of an angle near one
  radian, which moves sphere centres by about 1e-6 m, ten times the float32
  error of the GPU's positions).  A sample whose oracle gradient moves more
  than that (a sphere centre within about a millimetre of an obstacle's
  centre or axis, where the distance's direction turns quickly) is held to
  that movement instead, and counted.  Within the band the float32 positions
  decide the penetration depth itself, so the error there must stay below
  1e-3 of the gradient a penetration at the band's edge gives (2e-7); those
  samples are counted too.
Samples within reach of a kink of the distance (the oracle's central
differences at h and 2h disagree) are skipped and counted."""
import numpy as np
import pytest
import torch

import oracle
import vpgen

pytestmark = pytest.mark.gpu

MARGIN = 0.02
BAND = oracle.BAND  # 1e-4 m


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import CollisionCost, Validator, vp
    return Validator, CollisionCost, vp


def _kinky(o, q, margin):
    """Samples where FD at h and 2h disagree (near a kink)."""
    D = q.shape[1]
    bad = np.zeros(q.shape[0], dtype=bool)
    for h in (1e-6,):
        fd = []
        for hh in (h, 2 * h):
            Q = np.repeat(q[:, None, :], 2 * D, axis=1)
            for j in range(D):
                Q[:, 2 * j, j] += hh
                Q[:, 2 * j + 1, j] -= hh
            c = o.cost(Q.reshape(-1, D), margin, grad=False).reshape(-1, 2 * D)
            fd.append((c[:, 0::2] - c[:, 1::2]) / (2 * hh))
        scale = np.maximum(1.0, np.abs(fd[0]).max(axis=1))
        bad |= np.abs(fd[0] - fd[1]).max(axis=1) > 1e-6 * scale
    return bad


def _sensitivity(o, q, margin, g_ref, delta=1e-6, seed=0):
    """How far the oracle's gradient moves, relative to its largest
    component, when q moves by delta (two random directions, both signs)."""
    rng = np.random.default_rng(seed)
    scale = np.maximum(np.abs(g_ref).max(axis=1), 1e-300)
    s = np.zeros(q.shape[0])
    for _ in range(2):
        u = rng.uniform(-1.0, 1.0, size=q.shape)
        for sign in (1.0, -1.0):
            _, g = o.cost(q + sign * delta * u, margin)
            s = np.maximum(s, np.abs(g - g_ref).max(axis=1) / scale)
    return s


def _check(val, o, q, margin):
    """Check cost and gradient on every sample; returns (kink, band,
    sensitive, pinned) sample counts."""
    c_gpu, g_gpu = val.collision_cost(torch.from_numpy(q).cuda(), margin, grad=True)
    c_gpu, g_gpu = c_gpu.cpu().numpy().astype(np.float64), g_gpu.cpu().numpy().astype(np.float64)
    q64 = q.astype(np.float64)
    c_ref, g_ref = o.cost(q64, margin)
    np.testing.assert_allclose(c_gpu, c_ref, rtol=1e-4, atol=1e-6)
    kink = _kinky(o, q64, margin)
    sens = _sensitivity(o, q64, margin, g_ref)
    pen = np.sqrt(c_ref)
    outside = ~kink & (pen > BAND)
    pinned = outside & (sens <= 1e-3)
    sensitive = outside & ~pinned
    band = ~kink & ~outside
    scale = np.maximum(np.abs(g_ref).max(axis=1), 1e-300)
    err = np.abs(g_gpu - g_ref).max(axis=1)
    rel = err / scale
    assert np.all(rel[pinned] <= 1e-3), f"{int((rel[pinned] > 1e-3).sum())} samples, worst {rel[pinned].max():.3e}"
    assert np.all(rel[sensitive] <= sens[sensitive]), float((rel - sens)[sensitive].max())
    assert np.all(err[band] <= 1e-3 * 2 * BAND), float(err[band].max())
    print(f"{q.shape[0]} samples: {int(pinned.sum())} checked at relative 1e-3 (worst {rel[pinned].max():.2e}), "
          f"{int(sensitive.sum())} whose oracle gradient moves by more under a 1e-6 rad step (worst ratio "
          f"{(rel[sensitive] / sens[sensitive]).max() if sensitive.any() else 0:.2f}), "
          f"{int((band & (c_ref > 0)).sum())} penetrating within the band, {int(kink.sum())} near a kink")
    return int(kink.sum()), int(band.sum()), int(sensitive.sum()), int(pinned.sum())


def test_cost_and_gradient_mixed_scene(vpmod):
    """Every one of the 65,536 configurations of the mixed-primitive scene,
    and a 16,384-waypoint subset of its 4,096 straight 64-waypoint paths."""
    Validator, _, _ = vpmod
    w = vpgen.workload(vpgen.ARM7_MIXED128)
    val = Validator(w.robot, w.env)
    o = oracle.Oracle(w.robot, w.env)
    kinks, band, sensitive, pinned = _check(val, o, w.q0, MARGIN)
    assert kinks < 0.01 * w.q0.shape[0] and sensitive < 0.01 * w.q0.shape[0] and pinned > 0.3 * w.q0.shape[0]
    paths = vpgen.straight_paths(w.robot, 4096, 64, seed=303).reshape(-1, w.robot.dof)
    sub = paths[np.random.default_rng(303).choice(paths.shape[0], 16384, replace=False)]
    kinks, band, sensitive, pinned = _check(val, o, np.ascontiguousarray(sub), MARGIN)
    assert kinks < 0.01 * sub.shape[0] and sensitive < 0.01 * sub.shape[0] and pinned > 0.3 * sub.shape[0]


def test_gradient_tree_prismatic_general_axes(vpmod):
    """A branching robot with prismatic joints and general axes and origins
    exercises the subtree accumulation of the reverse sweep."""
    from robots_small import random_chain
    Validator, _, _ = vpmod
    rng = np.random.default_rng(12)
    r = random_chain(rng, D=9, n_spheres=40)
    r.joint_parent = np.array([-1, 0, 1, 2, 1, 4, -1, 6, 3], dtype=np.int32)
    env = vpgen.Env(np.array([[0.1, 0.1, 0.2, 0.3], [-0.2, 0.3, 0.0, 0.25]]),
                    np.array([[0.0, -0.3, 0.0, 0.3, 0.3, 0.3, 0.1]]),
                    np.array([np.concatenate([[0.2, 0.0, -0.1], np.eye(3).ravel(), [0.2, 0.15, 0.1]])]))
    val = Validator(r, env)
    o = oracle.Oracle(r, env)
    q = rng.uniform(-1.5, 1.5, size=(4096, 9)).astype(np.float32)
    kinks, band, sensitive, pinned = _check(val, o, q, MARGIN)
    assert kinks < 0.1 * q.shape[0] and sensitive < 0.01 * q.shape[0] and pinned > 0.3 * q.shape[0]


def test_cost_zero_and_no_grad(vpmod):
    Validator, _, _ = vpmod
    w = vpgen.workload(vpgen.ARM7_SPHERES16, n_edges=8)
    far = vpgen.Env(np.array([[50.0, 50, 50, 0.1]]), np.zeros((0, 7)), np.zeros((0, 15)))
    val = Validator(w.robot, far)
    c, g = val.collision_cost(torch.from_numpy(w.q0).cuda(), MARGIN, grad=True)
    assert float(c.abs().max()) == 0.0 and float(g.abs().max()) == 0.0
    c_only = val.collision_cost(torch.from_numpy(w.q0).cuda(), MARGIN, grad=False)
    assert c_only.shape == (8,)


def test_autograd_function(vpmod):
    Validator, CollisionCost, _ = vpmod
    w = vpgen.workload(vpgen.ARM7_MIXED128, n_edges=512)
    val = Validator(w.robot, w.env)
    q = torch.from_numpy(w.q0).cuda().requires_grad_(True)
    weights = torch.linspace(0.5, 1.5, 512, device="cuda")
    loss = (CollisionCost.apply(q, val, MARGIN) * weights).sum()
    loss.backward()
    _, g = val.collision_cost(q.detach(), MARGIN, grad=True)
    torch.testing.assert_close(q.grad, g * weights[:, None])


def test_path_repair_is_rejudged_by_the_boolean_check(vpmod):
    """Repair lowers the summed penetration cost of the waypoints, and the
    verdict of every repaired path comes from the boolean edge check (never
    from the cost): it equals an independent plain-mode check of its edges."""
    from paper_2309_14545_gb300.api import path_validity, repair_paths
    Validator, _, vp = vpmod
    r = vpgen.robot_for(vpgen.ARM7_MIXED128)
    env = vpgen.env_for(vpgen.ARM7_MIXED128)
    val = Validator(r, env)
    paths = torch.from_numpy(vpgen.straight_paths(r, 256, 64, seed=303)).cuda()
    inner = lambda p: p[:, 1:-1].reshape(-1, r.dof).contiguous()  # noqa: E731
    c0 = val.collision_cost(inner(paths), MARGIN).sum().item()
    fixed, before, after = repair_paths(val, paths, margin=MARGIN, iters=60, lr=0.02)
    c1 = val.collision_cost(inner(fixed), MARGIN).sum().item()
    assert c1 < 0.7 * c0
    assert torch.equal(after, path_validity(val, fixed, mode=vp.VP_MODE_PLAIN))
    assert torch.equal(fixed[:, 0], paths[:, 0]) and torch.equal(fixed[:, -1], paths[:, -1])
    assert bool((after | ~before).all()) and after.sum() >= before.sum()
