"""Seeded synthetic workloads for edge validation: robots, environments, edge sets.

This module holds no forward kinematics, distance, interpolation or validity
arithmetic: only seeded draws (NumPy PCG64 through ``default_rng``) and the
bookkeeping that lays them out as plain arrays.  Both the FP64 oracle and the
CUDA library read exactly these arrays, so no random-number generator has to
agree across languages.

Conventions shared by every consumer
------------------------------------
Robot (a forest of serial chains hanging off a fixed base):

* ``joint_parent[j]``  -1 (the base) or ``j - 1`` (the previous joint).
* ``joint_type[j]``    ``REVOLUTE`` (0) or ``PRISMATIC`` (1).
* ``joint_origin[j]``  fixed 3x4 ``[R | t]`` from the parent's frame to joint
  ``j``'s frame (before the joint moves).
* ``joint_axis[j]``    unit axis in joint ``j``'s frame.
* Link 0 is the base; link ``j + 1`` is the frame after joint ``j`` moved.
* ``sphere_link[s]``, ``sphere_centre[s]`` (in the link's frame),
  ``sphere_radius[s]``.
* ``link_spheres`` is ``None`` (the library derives one bounding sphere per
  link) or ``[n_links, 4]`` (centre in the link frame, radius; radius 0 for a
  link with no spheres).
* ``self_pairs[p] = (a, b)`` sphere indices checked against each other.

Environment: ``spheres [n,4]`` = centre, radius; ``capsules [n,7]`` = p0, p1,
radius; ``cuboids [n,15]`` = centre, R (3x3 row-major, columns are the box
axes in the world frame), half-extents.

Edges: ``q0, q1`` float32 ``[E, D]``; ``counts`` int32 ``[E]`` (explicit
state counts) or ``None`` (the count follows from ``res``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

REVOLUTE = 0
PRISMATIC = 1

#: Joint-space step of the validity-checking resolution (radians; the
#: prismatic joint's metres count the same, C-space being Euclidean).
RESOLUTION = np.float32(1.0 / 32.0)

#: Edge sets are drawn in fixed chunks so that any prefix is cheap and equal
#: to the same prefix of the full set.
EDGE_CHUNK = 65536

#: Workspace box in front of the base: x in [0.3, 1.3], y in [-0.5, 0.5],
#: z in [0, 1] (a 1 m cube 0.3 m in front of the base).
FRONT_BOX = ((0.3, 1.3), (-0.5, 0.5), (0.0, 1.0))
#: A 2 m cube centred at (1, 0, 1).
BIG_BOX = ((0.0, 2.0), (-1.0, 1.0), (0.0, 2.0))


@dataclass
class Robot:
    name: str
    joint_parent: np.ndarray
    joint_type: np.ndarray
    joint_axis: np.ndarray
    joint_origin: np.ndarray
    joint_lo: np.ndarray
    joint_hi: np.ndarray
    sphere_link: np.ndarray
    sphere_centre: np.ndarray
    sphere_radius: np.ndarray
    self_pairs: np.ndarray
    link_spheres: Optional[np.ndarray] = None
    # sphere centres in the world frame at q = 0, known from construction
    # (every generated chain is straight up at q = 0); used only to pick
    # self-collision pairs that are apart in that pose.
    rest_world: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def dof(self) -> int:
        return int(self.joint_type.shape[0])

    @property
    def n_links(self) -> int:
        return self.dof + 1

    @property
    def n_spheres(self) -> int:
        return int(self.sphere_radius.shape[0])


@dataclass
class Env:
    spheres: np.ndarray
    capsules: np.ndarray
    cuboids: np.ndarray

    @property
    def n_prims(self) -> int:
        return int(self.spheres.shape[0] + self.capsules.shape[0] + self.cuboids.shape[0])


@dataclass
class Workload:
    name: str
    robot: Robot
    env: Env
    q0: np.ndarray
    q1: np.ndarray
    counts: Optional[np.ndarray]
    res: np.float32
    margin: float = 0.0


# ----------------------------------------------------------------------------
# robots


def _translate(x, y, z):
    m = np.zeros((3, 4))
    m[:, :3] = np.eye(3)
    m[:, 3] = (x, y, z)
    return m


def _chain(rng, n_rev, n_spheres, base=(0.0, 0.0, 0.0), prismatic_torso=False, pedestal=False):
    """One serial chain: optional prismatic torso, then ``n_rev`` revolute joints.

    Link offsets are U[0.05, 0.35] m along the parent's z axis; revolute axes
    alternate z / y; limits are +-2.8 rad (torso 0..0.4 m).  Spheres (radius
    U[0.03, 0.08] m) are dealt round-robin over the chain's links and placed
    along each link's segment with +-0.02 m lateral jitter.

    Returns per-joint arrays (parent indices relative to the chain, -1 = base),
    per-link segment descriptions, and sphere tables with local link indices
    (0 = the chain's base/pedestal link when ``pedestal``).
    """
    types, axes, origins, lo, hi = [], [], [], [], []
    offsets = rng.uniform(0.05, 0.35, size=n_rev + 1)
    bx, by, bz = base
    # segment of each link in its own frame: (start z, end z) and the z of
    # the link frame's origin in the straight rest pose.
    seg = []  # list of (local z0, local z1, rest origin z)
    if pedestal:
        seg.append((-0.3, 0.0, bz))  # link 0 of the chain: the fixed base body
    z = bz
    if prismatic_torso:
        types.append(PRISMATIC)
        axes.append((0.0, 0.0, 1.0))
        origins.append(_translate(bx, by, bz))
        lo.append(0.0)
        hi.append(0.4)
        seg.append((0.0, offsets[0], z))
    for r in range(n_rev):
        types.append(REVOLUTE)
        axes.append((0.0, 0.0, 1.0) if r % 2 == 0 else (0.0, 1.0, 0.0))
        if r == 0 and not prismatic_torso:
            origins.append(_translate(bx, by, bz + offsets[0]))
        else:
            origins.append(_translate(0.0, 0.0, offsets[r]))
        z = z + offsets[r]
        lo.append(-2.8)
        hi.append(2.8)
        seg.append((0.0, offsets[r + 1], z))
    n_links_here = len(seg)
    sph_link = np.arange(n_spheres) % n_links_here
    t = rng.uniform(0.0, 1.0, size=n_spheres)
    jit = rng.uniform(-0.02, 0.02, size=(n_spheres, 2))
    rad = rng.uniform(0.03, 0.08, size=n_spheres)
    centre = np.zeros((n_spheres, 3))
    rest = np.zeros((n_spheres, 3))
    for s in range(n_spheres):
        z0, z1, zorg = seg[sph_link[s]]
        lz = z0 + t[s] * (z1 - z0)
        centre[s] = (jit[s, 0], jit[s, 1], lz)
        rest[s] = (bx + jit[s, 0], by + jit[s, 1], zorg + lz)
    # placement envelope of each link: every sphere of the link lies on the
    # segment, within 0.02*sqrt(2) laterally, with radius <= 0.08.
    env_sph = np.zeros((n_links_here, 4))
    for l, (z0, z1, _) in enumerate(seg):
        env_sph[l] = (0.0, 0.0, 0.5 * (z0 + z1), 0.5 * abs(z1 - z0) + 0.02 * np.sqrt(2.0) + 0.08)
    return dict(types=types, axes=axes, origins=origins, lo=lo, hi=hi,
                sph_link=sph_link, centre=centre, rad=rad, rest=rest,
                n_links_here=n_links_here, envelope=env_sph)


def _pick_pairs(rng, sphere_link, rest_world, radius, n_pairs, chain_of_link, link_gap=2, rest_clear=0.05):
    """Self-collision pairs: spheres on links at least ``link_gap`` apart within
    a chain (or on different chains) that are at least ``rest_clear`` m apart in
    the straight rest pose.  Drawn uniformly without replacement."""
    S = sphere_link.shape[0]
    cand = []
    for a in range(S):
        for b in range(a + 1, S):
            la, lb = sphere_link[a], sphere_link[b]
            if chain_of_link[la] == chain_of_link[lb] and abs(int(la) - int(lb)) < link_gap:
                continue
            gap = np.linalg.norm(rest_world[a] - rest_world[b]) - radius[a] - radius[b]
            if gap < rest_clear:
                continue
            cand.append((a, b))
    cand = np.array(cand, dtype=np.int32)
    idx = rng.choice(cand.shape[0], size=min(n_pairs, cand.shape[0]), replace=False)
    idx.sort()
    return cand[idx]


def arm7(seed: int = 0, n_spheres: int = 40) -> Robot:
    """7-DoF serial revolute arm, transforms from ``seed``; no self pairs."""
    rng = np.random.default_rng(seed)
    c = _chain(rng, 7, n_spheres)
    # chain links 0..6 are the frames after joints 0..6 = robot links 1..7
    return Robot(
        name=f"arm7-seed{seed}",
        joint_parent=np.array([-1] + list(range(6)), dtype=np.int32),
        joint_type=np.array(c["types"], dtype=np.int32),
        joint_axis=np.array(c["axes"], dtype=np.float64),
        joint_origin=np.array(c["origins"], dtype=np.float64),
        joint_lo=np.array(c["lo"]), joint_hi=np.array(c["hi"]),
        sphere_link=(c["sph_link"] + 1).astype(np.int32),
        sphere_centre=c["centre"], sphere_radius=c["rad"],
        self_pairs=np.zeros((0, 2), dtype=np.int32), link_spheres=None,
        rest_world=c["rest"],
    )


def torso_arm8(seed: int = 1, n_spheres: int = 100, n_pairs: int = 200) -> Robot:
    """8-DoF arm: prismatic torso (0..0.4 m) then 7 revolute joints.

    Spheres cover 9 links (the fixed pedestal, the torso and the 7 arm links);
    the 9 link bounding spheres are given (the placement envelope of each
    link), and 200 self pairs are drawn."""
    rng = np.random.default_rng(seed)
    c = _chain(rng, 7, n_spheres, prismatic_torso=True, pedestal=True)
    D = 8
    chain_of_link = np.zeros(D + 1, dtype=np.int32)
    pairs = _pick_pairs(rng, c["sph_link"], c["rest"], c["rad"], n_pairs, chain_of_link)
    return Robot(
        name=f"torso-arm8-seed{seed}",
        joint_parent=np.array([-1] + list(range(D - 1)), dtype=np.int32),
        joint_type=np.array(c["types"], dtype=np.int32),
        joint_axis=np.array(c["axes"], dtype=np.float64),
        joint_origin=np.array(c["origins"], dtype=np.float64),
        joint_lo=np.array(c["lo"]), joint_hi=np.array(c["hi"]),
        sphere_link=c["sph_link"].astype(np.int32),  # pedestal is chain link 0 = robot link 0
        sphere_centre=c["centre"], sphere_radius=c["rad"],
        self_pairs=pairs, link_spheres=c["envelope"].copy(),
        rest_world=c["rest"],
    )


def dual_arm14(n_spheres_per_arm: int = 60, n_pairs: int = 400, pair_seed: int = 2) -> Robot:
    """14-DoF dual arm: two 7-DoF chains (transforms from seeds 0 and 1) on a
    shared base, 0.5 m apart (y = +0.25 and y = -0.25)."""
    chains = []
    for seed, y in ((0, 0.25), (1, -0.25)):
        rng = np.random.default_rng(seed)
        chains.append(_chain(rng, 7, n_spheres_per_arm, base=(0.0, y, 0.0)))
    types, axes, origins, lo, hi, parent = [], [], [], [], [], []
    sl, sc, sr, rest = [], [], [], []
    for ci, c in enumerate(chains):
        j0 = len(types)
        types += c["types"]
        axes += c["axes"]
        origins += c["origins"]
        lo += c["lo"]
        hi += c["hi"]
        parent += [-1] + [j0 + r for r in range(6)]
        sl.append(c["sph_link"] + 1 + j0)
        sc.append(c["centre"])
        sr.append(c["rad"])
        rest.append(c["rest"])
    sphere_link = np.concatenate(sl).astype(np.int32)
    rest = np.concatenate(rest)
    rad = np.concatenate(sr)
    chain_of_link = np.array([0] + [1] * 7 + [2] * 7, dtype=np.int32)
    pairs = _pick_pairs(np.random.default_rng(pair_seed), sphere_link, rest, rad, n_pairs, chain_of_link)
    return Robot(
        name="dual-arm14",
        joint_parent=np.array(parent, dtype=np.int32),
        joint_type=np.array(types, dtype=np.int32),
        joint_axis=np.array(axes, dtype=np.float64),
        joint_origin=np.array(origins, dtype=np.float64),
        joint_lo=np.array(lo), joint_hi=np.array(hi),
        sphere_link=sphere_link, sphere_centre=np.concatenate(sc), sphere_radius=rad,
        self_pairs=pairs, link_spheres=None, rest_world=rest,
    )


# ----------------------------------------------------------------------------
# environments


def _uniform_in(rng, box, n):
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    return lo + (hi - lo) * rng.uniform(0.0, 1.0, size=(n, 3))


def _yaw_matrices(yaw):
    c, s = np.cos(yaw), np.sin(yaw)
    R = np.zeros((yaw.shape[0], 3, 3))
    R[:, 0, 0] = c
    R[:, 0, 1] = -s
    R[:, 1, 0] = s
    R[:, 1, 1] = c
    R[:, 2, 2] = 1.0
    return R


#: Keep-out columns above the robot bases: an obstacle whose axis-aligned
#: bounds enter |x - bx| <= 0.15, |y - by| <= 0.15, z <= 0.9 is redrawn, so no
#: obstacle overlaps a robot's fixed base (which would make every
#: configuration collide).
KEEPOUT_HALF = 0.15
KEEPOUT_TOP = 0.9
ARM_BASES = ((0.0, 0.0),)
DUAL_BASES = ((0.0, 0.25), (0.0, -0.25))


def _aabb(kind, p):
    """Axis-aligned bounds (lo[3], hi[3]) of one primitive row."""
    if kind == "sphere":
        return p[:3] - p[3], p[:3] + p[3]
    if kind == "capsule":
        return np.minimum(p[0:3], p[3:6]) - p[6], np.maximum(p[0:3], p[3:6]) + p[6]
    R = p[3:12].reshape(3, 3)
    ext = np.abs(R) @ p[12:15]
    return p[0:3] - ext, p[0:3] + ext


def _clear_of_bases(kind, p, bases):
    lo, hi = _aabb(kind, p)
    for bx, by in bases:
        if (lo[0] <= bx + KEEPOUT_HALF and hi[0] >= bx - KEEPOUT_HALF and
                lo[1] <= by + KEEPOUT_HALF and hi[1] >= by - KEEPOUT_HALF and lo[2] <= KEEPOUT_TOP):
            return False
    return True


def _draw(rng, n, one, kind, bases):
    """``n`` primitives from ``one(rng)``, each redrawn until clear of the bases."""
    rows = []
    while len(rows) < n:
        p = one(rng)
        if _clear_of_bases(kind, p, bases):
            rows.append(p)
    return np.array(rows).reshape(n, -1)


def _spheres(rng, box, n, bases, rlo=0.05, rhi=0.15):
    def one(g):
        return np.concatenate([_uniform_in(g, box, 1)[0], [g.uniform(rlo, rhi)]])
    return _draw(rng, n, one, "sphere", bases)


def _capsules(rng, box, n, bases):
    def one(g):
        p0 = _uniform_in(g, box, 1)[0]
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        length = g.uniform(0.1, 0.6)
        return np.concatenate([p0, p0 + d * length, [g.uniform(0.02, 0.08)]])
    return _draw(rng, n, one, "capsule", bases)


def _cuboids(rng, box, n, bases, hlo=0.02, hhi=0.4):
    def one(g):
        c = _uniform_in(g, box, 1)[0]
        R = _yaw_matrices(np.array([g.uniform(0.0, 2.0 * np.pi)]))[0]
        return np.concatenate([c, R.reshape(9), g.uniform(hlo, hhi, size=3)])
    return _draw(rng, n, one, "cuboid", bases)


def _empty(k):
    return np.zeros((0, k))


def env_spheres16(seed: int = 100) -> Env:
    rng = np.random.default_rng(seed)
    return Env(_spheres(rng, FRONT_BOX, 16, ARM_BASES), _empty(7), _empty(15))


def env_boxes_capsules(seed: int = 101) -> Env:
    rng = np.random.default_rng(seed)
    caps = _capsules(rng, FRONT_BOX, 20, ARM_BASES)
    return Env(_empty(4), caps, _cuboids(rng, FRONT_BOX, 60, ARM_BASES))


def env_shelves(seed: int = 102, n_total: int = 120, push: float = 0.0) -> Env:
    """Shelf-like scene of oriented cuboids: three shelf units around the
    front of the robot (uprights, back panel, five boards each) and small
    boxes standing on random boards.  Generated, not taken from any dataset.
    ``push`` moves every unit that far further from the robot."""
    rng = np.random.default_rng(seed)
    boxes = []

    def add(centre, yaw, half):
        R = _yaw_matrices(np.array([yaw]))[0]
        boxes.append(np.concatenate([np.asarray(centre, float), R.reshape(9), np.asarray(half, float)]))

    units = [((0.85 + push, 0.0), 0.0), ((0.2, 0.95 + push), np.pi / 2), ((0.2, -0.95 - push), -np.pi / 2)]
    depth, width, height = 0.35, 0.9, 1.6
    levels = [0.25, 0.55, 0.85, 1.15, 1.45]
    boards = []
    for (cx, cy), yaw in units:
        R = _yaw_matrices(np.array([yaw]))[0]
        ax_d, ax_w = R[:, 0], R[:, 1]  # unit's depth and width directions in the world
        base = np.array([cx, cy, 0.0])
        for side in (-1, 1):
            c = base + ax_w * side * (width / 2) + np.array([0, 0, height / 2])
            add(c, yaw, (depth / 2, 0.01, height / 2))
        add(base + ax_d * (depth / 2) + np.array([0, 0, height / 2]), yaw, (0.01, width / 2, height / 2))
        for z in levels:
            add(base + np.array([0, 0, z]), yaw, (depth / 2, width / 2, 0.01))
            boards.append((base, ax_d, ax_w, z, yaw))
    n_obj = n_total - len(boxes)
    pick = rng.integers(0, len(boards), size=n_obj)
    for i in range(n_obj):
        base, ax_d, ax_w, z, yaw = boards[pick[i]]
        half = rng.uniform(0.02, 0.06, size=3)
        u = rng.uniform(-0.12, 0.12)
        v = rng.uniform(-0.4, 0.4)
        c = base + ax_d * u + ax_w * v + np.array([0, 0, z + 0.01 + half[2]])
        add(c, yaw + rng.uniform(0, 2 * np.pi), half)
    return Env(_empty(4), _empty(7), np.array(boxes))


def env_mixed128(seed: int = 103) -> Env:
    rng = np.random.default_rng(seed)
    sph = _spheres(rng, FRONT_BOX, 64, ARM_BASES)
    caps = _capsules(rng, FRONT_BOX, 32, ARM_BASES)
    return Env(sph, caps, _cuboids(rng, FRONT_BOX, 32, ARM_BASES))


def env_mixed1000(seed: int = 104, shift: float = 0.0) -> Env:
    """1,000 primitives in the 2 m cube centred at (1 + shift, 0, 1)."""
    rng = np.random.default_rng(seed)
    box = ((BIG_BOX[0][0] + shift, BIG_BOX[0][1] + shift), BIG_BOX[1], BIG_BOX[2])
    sph = _spheres(rng, box, 400, DUAL_BASES)
    caps = _capsules(rng, box, 300, DUAL_BASES)
    return Env(sph, caps, _cuboids(rng, box, 300, DUAL_BASES))


# ----------------------------------------------------------------------------
# edge sets


def uniform_configs(robot: Robot, n: int, seed: int) -> np.ndarray:
    """``n`` configurations uniform within the joint limits, as float32,
    drawn in chunks of ``EDGE_CHUNK`` (any prefix equals the full draw's)."""
    D = robot.dof
    out = np.empty((n, D), dtype=np.float32)
    lo, hi = robot.joint_lo, robot.joint_hi
    for c0 in range(0, n, EDGE_CHUNK):
        m = min(EDGE_CHUNK, n - c0)
        rng = np.random.default_rng([seed, c0 // EDGE_CHUNK])
        out[c0:c0 + m] = (lo + (hi - lo) * rng.uniform(0.0, 1.0, size=(m, D))).astype(np.float32)
    return out


def uniform_edges(robot: Robot, n: int, seed: int):
    """Edge endpoints uniform within the limits: (q0, q1) float32 [n, D]."""
    D = robot.dof
    q0 = np.empty((n, D), dtype=np.float32)
    q1 = np.empty((n, D), dtype=np.float32)
    lo, hi = robot.joint_lo, robot.joint_hi
    for c0 in range(0, n, EDGE_CHUNK):
        m = min(EDGE_CHUNK, n - c0)
        rng = np.random.default_rng([seed, c0 // EDGE_CHUNK])
        u = rng.uniform(0.0, 1.0, size=(2, m, D))
        q0[c0:c0 + m] = (lo + (hi - lo) * u[0]).astype(np.float32)
        q1[c0:c0 + m] = (lo + (hi - lo) * u[1]).astype(np.float32)
    return q0, q1


def mid_edges(robot: Robot, n: int, seed: int, span: float = 0.5):
    """Edge endpoints uniform within the middle ``span`` of each joint's
    range, around its midpoint (configurations nearer a home pose, where a
    two-arm robot is mostly clear of itself): (q0, q1) float32 [n, D],
    drawn in chunks like ``uniform_edges``."""
    D = robot.dof
    q0 = np.empty((n, D), dtype=np.float32)
    q1 = np.empty((n, D), dtype=np.float32)
    lo, hi = robot.joint_lo, robot.joint_hi
    mid, half = 0.5 * (lo + hi), 0.5 * span * (hi - lo)
    for c0 in range(0, n, EDGE_CHUNK):
        m = min(EDGE_CHUNK, n - c0)
        rng = np.random.default_rng([seed, 5, c0 // EDGE_CHUNK])
        u = rng.uniform(-1.0, 1.0, size=(2, m, D))
        q0[c0:c0 + m] = (mid + half * u[0]).astype(np.float32)
        q1[c0:c0 + m] = (mid + half * u[1]).astype(np.float32)
    return q0, q1


def loguniform_counts(n: int, seed: int, kmin: int = 2, kmax: int = 512) -> np.ndarray:
    """Explicit per-edge state counts, round(exp(U[ln kmin, ln kmax]))."""
    out = np.empty(n, dtype=np.int32)
    for c0 in range(0, n, EDGE_CHUNK):
        m = min(EDGE_CHUNK, n - c0)
        rng = np.random.default_rng([seed, 7, c0 // EDGE_CHUNK])
        out[c0:c0 + m] = np.rint(np.exp(rng.uniform(np.log(kmin), np.log(kmax), size=m))).astype(np.int32)
    return np.clip(out, kmin, kmax)


def straight_paths(robot: Robot, n_paths: int, n_way: int, seed: int) -> np.ndarray:
    """``n_paths`` straight joint-space paths of ``n_way`` evenly spaced
    waypoints between random endpoints: float32 [n_paths, n_way, D]."""
    qa, qb = uniform_edges(robot, n_paths, seed)
    s = (np.arange(n_way, dtype=np.float64) / (n_way - 1))[None, :, None]
    w = qa.astype(np.float64)[:, None, :] + s * (qb.astype(np.float64) - qa.astype(np.float64))[:, None, :]
    return w.astype(np.float32)


def jagged_paths(robot: Robot, n_paths: int, n_way: int, seed: int, span: float = 0.5,
                 noise: float = 0.25) -> np.ndarray:
    """Jagged joint-space paths, the raw output a sampling planner leaves for
    shortcutting: ``n_way`` waypoints evenly spaced between random endpoints
    (drawn within ``span`` of the joint range around its middle), interior
    waypoints displaced by U[-noise, noise] rad per joint, clipped to the
    limits.  float32 [n_paths, n_way, D]."""
    D = robot.dof
    lo, hi = robot.joint_lo, robot.joint_hi
    mid, half = 0.5 * (lo + hi), 0.5 * span * (hi - lo)
    rng = np.random.default_rng([seed, 7])
    a = mid + half * rng.uniform(-1.0, 1.0, size=(n_paths, D))
    b = mid + half * rng.uniform(-1.0, 1.0, size=(n_paths, D))
    s = (np.arange(n_way, dtype=np.float64) / (n_way - 1))[None, :, None]
    w = a[:, None, :] + s * (b - a)[:, None, :]
    jitter = rng.uniform(-noise, noise, size=(n_paths, n_way, D))
    jitter[:, 0] = 0.0
    jitter[:, -1] = 0.0
    return np.clip(w + jitter, lo, hi).astype(np.float32)


def shortcut_draws(n_iter: int, n_paths: int, seed: int) -> np.ndarray:
    """The random numbers randomized shortcutting consumes: U[0, 1) float32
    [n_iter, n_paths, 2] (two waypoint positions per path and iteration)."""
    rng = np.random.default_rng([seed, 11])
    return rng.uniform(0.0, 1.0, size=(n_iter, n_paths, 2)).astype(np.float32)


def rrt_problems(robot: Robot, n_problems: int, n_samples: int, seed: int):
    """Planning problems for batched RRT-Connect: start and goal uniform in
    the limits, and each problem's own ``n_samples`` uniform configurations
    (the random draws the planner consumes).  float32 ([B, D], [B, D],
    [B, T, D])."""
    start, goal = uniform_edges(robot, n_problems, seed)
    D = robot.dof
    lo, hi = robot.joint_lo, robot.joint_hi
    rng = np.random.default_rng([seed, 13])
    samples = (lo + (hi - lo) * rng.uniform(0.0, 1.0, size=(n_problems, n_samples, D))).astype(np.float32)
    return start, goal, samples


#: RRT-Connect workloads: (robot/scene workload, problems, samples each,
#: range in rad, tree capacity).
RRT_CASES = (("arm7_spheres16", 4096, 1024, 1.0, 1024),
             ("torso8_obb60_cap20", 2048, 1024, 0.8, 1024))
RRT_SEED = 307

#: Shortcutting workload: the 7-DoF arm among the 16-sphere scene
#: (``arm7_spheres16``), 4,096 jagged paths of 32 waypoints, 64 iterations.
SHORTCUT_PATHS, SHORTCUT_WAYPOINTS, SHORTCUT_ITERS, SHORTCUT_SEED = 4096, 32, 64, 305


# ----------------------------------------------------------------------------
# the workloads, by name

ARM7_SPHERES16 = "arm7_spheres16"          # 7-DoF arm vs 16 spheres, 10,000 edges
TORSO8_OBB60_CAP20 = "torso8_obb60_cap20"  # 8-DoF torso arm vs 60 OBBs + 20 capsules, 1,000,000 edges
DUAL14_SHELVES = "dual14_shelves"          # 14-DoF dual arm vs 120-cuboid shelves, 262,144 edges
ARM7_MIXED128 = "arm7_mixed128"            # 7-DoF arm vs 128 mixed primitives, 65,536 configurations
DUAL14_MIXED1000 = "dual14_mixed1000"      # 14-DoF dual arm vs 1,000 mixed primitives, 4,194,304 edges
# Obstacle-shifted variants of the two dual-arm workloads (same robot, same
# edges and counts; only the obstacles move away), added because random
# edges there are almost all invalid.  Self contact between the two arms
# already leaves only ~2.7% of those edges collision-free, which bounds any
# obstacle placement.
DUAL14_SHELVES_FAR = "dual14_shelves_far"      # shelves pushed 0.6 m further out
DUAL14_MIXED1000_FAR = "dual14_mixed1000_far"  # the 2 m cube centred 1 m further out
# Variants with mostly collision-free edges, so that the costly case -- every
# state of a long edge checked against the whole scene -- is timed and
# checked too: endpoints in the middle half of each joint's range (``mid``).
# The shelves stay where they are (about 11% of these edges are valid); the
# 1,000 primitives are those of the far variant (about 38% valid), since in
# the base cube even these configurations almost all touch an obstacle.
DUAL14_SHELVES_MID = "dual14_shelves_mid"
DUAL14_MIXED1000_MID = "dual14_mixed1000_mid"
NAMES = (ARM7_SPHERES16, TORSO8_OBB60_CAP20, DUAL14_SHELVES, ARM7_MIXED128, DUAL14_MIXED1000, DUAL14_SHELVES_FAR,
         DUAL14_MIXED1000_FAR, DUAL14_SHELVES_MID, DUAL14_MIXED1000_MID)
_VARIANT_OF = {DUAL14_SHELVES_FAR: DUAL14_SHELVES, DUAL14_MIXED1000_FAR: DUAL14_MIXED1000}

#: Full sizes of the workloads.
FULL_EDGES = {ARM7_SPHERES16: 10_000, TORSO8_OBB60_CAP20: 1_000_000, DUAL14_SHELVES: 262_144,
              ARM7_MIXED128: 65_536, DUAL14_MIXED1000: 4_194_304, DUAL14_SHELVES_FAR: 262_144,
              DUAL14_MIXED1000_FAR: 4_194_304, DUAL14_SHELVES_MID: 262_144, DUAL14_MIXED1000_MID: 4_194_304}

DESCRIPTION = {
    ARM7_SPHERES16: "7-DoF arm (40 spheres) vs 16 spheres; 10,000 uniform edges at 1/32 rad",
    TORSO8_OBB60_CAP20: "8-DoF torso arm (100 spheres / 9 links / 200 self pairs) vs 60 OBBs + 20 capsules; "
                        "1,000,000 edges at 1/32 rad",
    DUAL14_SHELVES: "14-DoF dual arm (120 spheres / 400 self pairs) vs 120-cuboid shelves; 262,144 edges, "
                    "counts log-uniform in [2,512]",
    ARM7_MIXED128: "7-DoF arm vs 64 spheres + 32 capsules + 32 OBBs; cost at margin 0.02 on 65,536 configurations",
    DUAL14_MIXED1000: "14-DoF dual arm vs 1,000 mixed primitives in a 2 m cube; 4,194,304 edges, counts "
                      "log-uniform in [2,512]",
    DUAL14_SHELVES_FAR: "dual14_shelves with the shelf units 0.6 m further out (same edges)",
    DUAL14_MIXED1000_FAR: "dual14_mixed1000 with the 2 m cube centred 1 m further out (same edges)",
    DUAL14_SHELVES_MID: "dual14_shelves scene; 262,144 edges between configurations in the middle half of each "
                        "joint range, counts log-uniform in [2,512]",
    DUAL14_MIXED1000_MID: "dual14_mixed1000_far scene (1,000 primitives, cube centred at (2, 0, 1)); 4,194,304 "
                          "edges between configurations in the middle half of each joint range, counts "
                          "log-uniform in [2,512]",
}

# seeds: robots 0/1/2; scenes 100 + index; edges 200 + index (index = position in NAMES)
_INDEX = {n: i for i, n in enumerate(NAMES)}


def robot_for(name: str) -> Robot:
    if name in (ARM7_SPHERES16, ARM7_MIXED128):
        return arm7(0, 40)
    if name == TORSO8_OBB60_CAP20:
        return torso_arm8(1, 100, 200)
    if name in (DUAL14_SHELVES, DUAL14_MIXED1000, DUAL14_SHELVES_FAR, DUAL14_MIXED1000_FAR, DUAL14_SHELVES_MID,
                DUAL14_MIXED1000_MID):
        return dual_arm14(60, 400)
    raise ValueError(name)


def env_for(name: str) -> Env:
    return {ARM7_SPHERES16: env_spheres16, TORSO8_OBB60_CAP20: env_boxes_capsules, DUAL14_SHELVES: env_shelves,
            ARM7_MIXED128: env_mixed128, DUAL14_MIXED1000: env_mixed1000,
            DUAL14_SHELVES_FAR: lambda: env_shelves(push=0.6),
            DUAL14_MIXED1000_FAR: lambda: env_mixed1000(shift=1.0), DUAL14_SHELVES_MID: env_shelves,
            DUAL14_MIXED1000_MID: lambda: env_mixed1000(shift=1.0)}[name]()


def workload(name: str, n_edges: Optional[int] = None, robot: Optional[Robot] = None,
             env: Optional[Env] = None) -> Workload:
    """Workload ``name`` with its first ``n_edges`` edges (default: all).

    ``arm7_mixed128`` is a configuration set, returned as ``q0 == q1`` edges
    with ``margin = 0.02``."""
    if name not in _INDEX:
        raise ValueError(f"unknown workload {name!r}; one of {NAMES}")
    robot = robot if robot is not None else robot_for(name)
    env = env if env is not None else env_for(name)
    n = FULL_EDGES[name] if n_edges is None else int(n_edges)
    if name in _VARIANT_OF:  # the base workload's edges, the variant's obstacles
        base = workload(_VARIANT_OF[name], n_edges=n, robot=robot, env=env)
        base.name = name
        return base
    seed = 200 + _INDEX[name]
    if name in (ARM7_SPHERES16, TORSO8_OBB60_CAP20):
        q0, q1 = uniform_edges(robot, n, seed)
        return Workload(name, robot, env, q0, q1, None, RESOLUTION)
    if name in (DUAL14_SHELVES, DUAL14_MIXED1000):
        q0, q1 = uniform_edges(robot, n, seed)
        return Workload(name, robot, env, q0, q1, loguniform_counts(n, seed), RESOLUTION)
    if name in (DUAL14_SHELVES_MID, DUAL14_MIXED1000_MID):
        q0, q1 = mid_edges(robot, n, seed)
        return Workload(name, robot, env, q0, q1, loguniform_counts(n, seed), RESOLUTION)
    q = uniform_configs(robot, n, seed)
    return Workload(name, robot, env, q, q.copy(), None, RESOLUTION, margin=0.02)
