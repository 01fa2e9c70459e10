"""Per-robot FK by code generation (vp_fk_codegen) against the table-driven
FK kernel and the FP64 oracle.  The generated kernel computes what the
table-driven one computes in the same order of operations (zero terms
dropped, which is exact for finite frames), so the two agree to within a
unit of rounding; both stay within 1e-5 m of the oracle."""
import numpy as np
import pytest
import torch

import oracle
import vpgen
from robots_small import EMPTY_ENV, random_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vpmod(cuda_ok):
    from paper_2309_14545_gb300 import build
    build.build()
    from paper_2309_14545_gb300 import Validator, vp
    return Validator, vp


def _tree():
    rng = np.random.default_rng(12)
    r = random_chain(rng, D=9, n_spheres=40)
    r.joint_parent = np.array([-1, 0, 1, 2, 1, 4, -1, 6, 3], dtype=np.int32)
    return r


@pytest.mark.parametrize("make", [lambda: vpgen.robot_for(vpgen.ARM7_SPHERES16),
                                  lambda: vpgen.robot_for(vpgen.TORSO8_OBB60_CAP20),
                                  lambda: vpgen.robot_for(vpgen.DUAL14_SHELVES),
                                  lambda: random_chain(np.random.default_rng(4), D=6, n_spheres=30),
                                  _tree])
def test_generated_fk_matches_table_and_oracle(vpmod, make):
    Validator, vp = vpmod
    r = make()
    val = Validator(r, EMPTY_ENV)
    q = torch.from_numpy(vpgen.uniform_configs(r, 4099, seed=8)).cuda()
    default = val.fk_spheres(q).cpu().numpy()  # the automatic choice: the generated kernel
    val.fk_codegen(False)
    table = val.fk_spheres(q).cpu().numpy()
    ms = val.fk_codegen(True)
    assert ms > 0
    gen = val.fk_spheres(q).cpu().numpy()
    assert np.array_equal(gen, default)
    val.fk_codegen(False)
    again = val.fk_spheres(q).cpu().numpy()
    assert np.array_equal(again, table)  # switched back to the table
    val.fk_codegen(-1)
    assert np.array_equal(val.fk_spheres(q).cpu().numpy(), gen)
    with pytest.raises(vp.VPError):
        val.fk_codegen(2)
    assert np.abs(gen - table).max() <= 4e-7 * max(1.0, np.abs(table).max())
    want = oracle.Oracle(r, EMPTY_ENV).fk(q.cpu().numpy().astype(np.float64))
    assert np.abs(gen - want).max() < 1e-5
    val.close()


def test_reloading_the_robot_drops_the_generated_kernel(vpmod):
    Validator, vp = vpmod
    a, b = vpgen.robot_for(vpgen.ARM7_SPHERES16), random_chain(np.random.default_rng(5), D=7, n_spheres=40)
    val = Validator(a, EMPTY_ENV)
    val.fk_codegen(True)
    vp.vp_load_robot(val.ctx, b)
    q = torch.from_numpy(vpgen.uniform_configs(b, 257, seed=2)).cuda()
    out = torch.empty((257, 40, 3), dtype=torch.float32, device="cuda")
    vp.vp_fk_spheres(val.ctx, q, out)
    want = oracle.Oracle(b, EMPTY_ENV).fk(q.cpu().numpy().astype(np.float64))
    assert np.abs(out.cpu().numpy() - want).max() < 1e-5
    val.close()


def test_generated_fk_ragged_and_unaligned_output(vpmod):
    """Both FK kernels write each block's rows with one bulk copy.  An odd
    sphere count leaves a last block whose bytes are not a multiple of 16
    (the remainder goes by plain stores), and an output that starts off a
    16-byte boundary takes plain stores only: both give the same centres."""
    Validator, vp = vpmod
    S, N = 13, 4099
    r = random_chain(np.random.default_rng(6), D=5, n_spheres=S)
    val = Validator(r, EMPTY_ENV)
    q = torch.from_numpy(vpgen.uniform_configs(r, N, seed=3)).cuda()
    table = val.fk_spheres(q).cpu().numpy()
    raw_t = torch.zeros(N * S * 3 + 1, dtype=torch.float32, device="cuda")
    vp.vp_fk_spheres(val.ctx, q, raw_t[1:].view(N, S, 3))
    assert np.array_equal(raw_t[1:].view(N, S, 3).cpu().numpy(), table) and raw_t[0].item() == 0.0
    val.fk_codegen(True)
    gen = val.fk_spheres(q).cpu().numpy()
    assert np.abs(gen - table).max() <= 4e-7 * max(1.0, np.abs(table).max())
    want = oracle.Oracle(r, EMPTY_ENV).fk(q.cpu().numpy().astype(np.float64))
    assert np.abs(gen - want).max() < 1e-5
    raw = torch.zeros(N * S * 3 + 1, dtype=torch.float32, device="cuda")
    shifted = raw[1:].view(N, S, 3)
    assert shifted.data_ptr() % 16 != 0
    vp.vp_fk_spheres(val.ctx, q, shifted)
    assert np.array_equal(shifted.cpu().numpy(), gen)
    assert raw[0].item() == 0.0
    val.close()
