"""Build libvp.so (the CUDA library behind include/vp.h) in-tree with nvcc.

Every translation unit is compiled for sm_103a only, in parallel, then
linked into ``paper_2309_14545_gb300/libvp.so``.  No fast-math: the
kernels rely on IEEE division and accurate ``sincosf``.
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libvp.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "128"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(cuda, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _deps():
    return glob.glob(os.path.join(CSRC, "*")) + [os.path.join(HERE, "..", "include", "vp.h")]


# The files that define the edge-validation kernels (device code, tables and
# their layouts); host-side launch code, the tuner and other kernels are not.
KERNEL_FILES = ("vp_types.h", "vp_device.cuh", "vp_validate.cuh", "vp_batched.h", "vp_batched.cu", "vp_inst.cu",
                "vp_api.cu")

# vp_inst.cu holds the validation kernels of one link bound and one family of
# check orders per compilation: it is compiled once for each pair.
INST_LMAX = (8, 9, 15, 17)
INST_FAMILIES = (0, 1, 2)


def _code_only(text: str) -> str:
    """The source with its comments and runs of whitespace removed, so that
    edits to comments and layout leave the hash unchanged."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash() -> str:
    """Hash of the code (comments and whitespace aside) of the
    edge-validation kernels, the packer that builds their tables (vp_api.cu)
    and the public header: counters measured on one build
    (profiles/traffic.json) apply to another with the same hash."""
    import hashlib
    h = hashlib.sha256()
    for p in [os.path.join(CSRC, f) for f in KERNEL_FILES] + [os.path.join(HERE, "..", "include", "vp.h")]:
        h.update(os.path.basename(p).encode())
        h.update(_code_only(open(p, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libvp.so unless it is newer than every source."""
    if not force and up_to_date():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    inst = os.path.join(CSRC, "vp_inst.cu")
    units = [(p, ()) for p in sorted(glob.glob(os.path.join(CSRC, "*.cu"))) if p != inst]
    units += [(inst, (f"-DVP_INST_LMAX={l}", f"-DVP_INST_FAM={f}")) for l in INST_LMAX for f in INST_FAMILIES]
    # the slowest units first, so that they start at once
    units.sort(key=lambda u: (u[0] != inst, u[0]))
    nvcc = _nvcc()

    def compile_one(unit):
        src, defs = unit
        tag = os.path.basename(src) + "".join(d.split("=")[-1] for d in defs)
        obj = os.path.join(BUILD, tag + f".{os.getpid()}.o")
        cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(units), max(4, os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = OUT + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
