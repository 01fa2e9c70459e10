"""The C-ABI library builds, loads and exports every symbol include/vp.h
declares; the Python binding mirrors those names.  No compute calls here
(CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vp.h")).read()
    return set(re.findall(r"^(?:vp_status|const char \*)\s*(vp_\w+)\s*\(", src, re.M))


@pytest.fixture(scope="module")
def libpath():
    from paper_2309_14545_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("vp_load_robot", "vp_load_env", "vp_validate_states", "vp_validate_edges", "vp_collision_cost"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(vp_\w+)$", out, re.M))
    missing = _declared() - exported
    assert not missing, missing


def test_binding_mirrors_the_header(libpath):
    from paper_2309_14545_gb300 import vp
    assert set(vp.EXPORTS) == _declared()
    for n in vp.EXPORTS:
        assert callable(getattr(vp, n))
        assert getattr(vp.lib, n) is not None


def test_header_constants_match_binding():
    from paper_2309_14545_gb300 import vp
    src = open(os.path.join(ROOT, "include", "vp.h")).read()
    consts = {k: v.strip() for k, v in re.findall(r"#define (VP_\w+) \(?([0-9a-fx*u ]+)", src)}
    assert int(consts["VP_MAX_JOINTS"]) == vp.VP_MAX_JOINTS
    assert int(consts["VP_MAX_SPHERES"]) == vp.VP_MAX_SPHERES
    assert int(consts["VP_MAX_PAIRS"]) == vp.VP_MAX_PAIRS
    assert int(consts["VP_MAX_STEPS"]) == vp.VP_MAX_STEPS
    assert eval(consts["VP_MAX_ENV_BYTES"]) == vp.VP_MAX_ENV_BYTES
    assert int(consts["VP_DEVERR_COUNT"].rstrip("u"), 16) == vp.VP_DEVERR_COUNT
    assert int(consts["VP_DEVERR_TIMEOUT"].rstrip("u"), 16) == vp.VP_DEVERR_TIMEOUT


def test_create_without_a_device_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2309_14545_gb300 import vp
    with pytest.raises(vp.VPError):
        vp.vp_create(0)


def test_product_path_does_not_touch_the_oracle():
    """The package never imports, links or runs anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2309_14545_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                for needle in ("import oracle", "from oracle", "liboracle", "vp_oracle", "vpo_"):
                    assert needle not in text, (f, needle)
