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
KERNEL_FILES = ("vp_types.h", "vp_device.cuh", "vp_validate.cuh", "vp_batched.h", "vp_inst_l8.cu", "vp_inst_l9.cu",
                "vp_inst_l15.cu", "vp_inst_l17.cu", "vp_api.cu")


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
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + f".{os.getpid()}.o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
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
