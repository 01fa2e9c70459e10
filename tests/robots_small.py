"""Tiny hand-built robots and scenes for pinning the oracle (test helpers)."""
import numpy as np

import vpgen


def _rt(R=None, t=(0.0, 0.0, 0.0)):
    m = np.zeros((3, 4))
    m[:, :3] = np.eye(3) if R is None else R
    m[:, 3] = t
    return m


def planar2(L1=0.7, L2=0.4, r=0.05):
    """Planar 2-link arm in the xy plane: both joints about z, joint 2 at
    (L1, 0, 0) in link 1's frame; spheres at the elbow (link 1, (L1,0,0))
    and at the tip (link 2, (L2,0,0))."""
    return vpgen.Robot(
        name="planar2",
        joint_parent=np.array([-1, 0], dtype=np.int32),
        joint_type=np.array([vpgen.REVOLUTE, vpgen.REVOLUTE], dtype=np.int32),
        joint_axis=np.array([[0, 0, 1.0], [0, 0, 1.0]]),
        joint_origin=np.array([_rt(), _rt(t=(L1, 0, 0))]),
        joint_lo=np.array([-np.pi, -np.pi]), joint_hi=np.array([np.pi, np.pi]),
        sphere_link=np.array([1, 2], dtype=np.int32),
        sphere_centre=np.array([[L1, 0, 0], [L2, 0, 0.0]]),
        sphere_radius=np.array([r, r]),
        self_pairs=np.zeros((0, 2), dtype=np.int32),
    )


def one_joint(jtype, axis, origin_R=None, origin_t=(0, 0, 0), local=(0.3, -0.2, 0.5), r=0.05):
    return vpgen.Robot(
        name="one",
        joint_parent=np.array([-1], dtype=np.int32),
        joint_type=np.array([jtype], dtype=np.int32),
        joint_axis=np.array([axis], dtype=np.float64),
        joint_origin=np.array([_rt(origin_R, origin_t)]),
        joint_lo=np.array([-3.0]), joint_hi=np.array([3.0]),
        sphere_link=np.array([1, 0], dtype=np.int32),
        sphere_centre=np.array([local, (0.1, 0.2, 0.3)], dtype=np.float64),
        sphere_radius=np.array([r, r]),
        self_pairs=np.zeros((0, 2), dtype=np.int32),
    )


def random_chain(rng, D=5, n_spheres=12, general=True):
    """Serial chain with random fixed rotations and random unit axes."""
    from scipy.spatial.transform import Rotation
    origins = []
    axes = []
    for j in range(D):
        R = Rotation.from_rotvec(rng.normal(size=3)).as_matrix() if general else np.eye(3)
        origins.append(_rt(R, rng.uniform(-0.3, 0.3, size=3)))
        a = rng.normal(size=3)
        axes.append(a / np.linalg.norm(a))
    types = rng.integers(0, 2, size=D).astype(np.int32)
    return vpgen.Robot(
        name="random-chain",
        joint_parent=np.arange(-1, D - 1, dtype=np.int32),
        joint_type=types,
        joint_axis=np.array(axes),
        joint_origin=np.array(origins),
        joint_lo=np.full(D, -2.0), joint_hi=np.full(D, 2.0),
        sphere_link=rng.integers(0, D + 1, size=n_spheres).astype(np.int32),
        sphere_centre=rng.uniform(-0.2, 0.2, size=(n_spheres, 3)),
        sphere_radius=rng.uniform(0.02, 0.06, size=n_spheres),
        self_pairs=np.zeros((0, 2), dtype=np.int32),
    )


EMPTY_ENV = vpgen.Env(np.zeros((0, 4)), np.zeros((0, 7)), np.zeros((0, 15)))


def env_of(spheres=(), capsules=(), cuboids=()):
    return vpgen.Env(np.array(spheres, dtype=np.float64).reshape(-1, 4),
                     np.array(capsules, dtype=np.float64).reshape(-1, 7),
                     np.array(cuboids, dtype=np.float64).reshape(-1, 15))


def cuboid_row(c, R, h):
    return np.concatenate([np.asarray(c, float), np.asarray(R, float).reshape(9), np.asarray(h, float)])
