"""Builds libsz3g.so in-tree from csrc/*.cu for sm_103a (nvcc only, no cmake).

Every translation unit is compiled in parallel; the library links the CUDA
runtime statically so it loads next to any PyTorch build.  Floating point is
compiled strictly: no fused multiply-add contraction (-fmad=false), IEEE
division and square root, no flush-to-zero -- the prediction and quantizer
steps must round exactly as written.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_obj")
LIB = os.path.join(HERE, "libsz3g.so")
# the checking build: every kernel index check compiled in (SZ3G_CHECK)
OBJ_CHECK = os.path.join(HERE, "_obj_check")
LIB_CHECK = os.path.join(HERE, "libsz3g_check.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false",
    "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills", f"-I{INCLUDE}",
]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stamp() -> str:
    """Hash of the sources, the public header and the compile flags, keyed by
    names relative to the package so that a copy of the tree elsewhere gives
    the same stamp."""
    h = hashlib.sha256()
    files = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "sz3g.h")]
    for p in files:
        with open(p, "rb") as fh:
            h.update(os.path.relpath(p, os.path.dirname(HERE)).encode() + fh.read())
    h.update(" ".join(f for f in NVCC_FLAGS if not f.startswith("-I")).encode())
    return h.hexdigest()


# The sources each measured kernel is compiled and launched from (its own
# file, the headers it includes, the plan that sizes its work).
KERNEL_SOURCES = {
    "level_quantize": ["k_fine.cu", "level_common.cuh", "internal.cuh", "plan.cu"],
    "level_recover": ["k_fine.cu", "level_common.cuh", "internal.cuh", "plan.cu"],
}


def kernel_stamp(kernel: str) -> str:
    """Hash of the sources of one measured kernel, the public header and the
    compile flags: a counter taken on a kernel stays valid while this holds."""
    h = hashlib.sha256()
    files = [os.path.join(CSRC, f) for f in KERNEL_SOURCES[kernel]] + [os.path.join(INCLUDE, "sz3g.h")]
    for p in files:
        with open(p, "rb") as fh:
            h.update(os.path.relpath(p, os.path.dirname(HERE)).encode() + fh.read())
    h.update(" ".join(f for f in NVCC_FLAGS if not f.startswith("-I")).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Builds the library (or, check=True, the checking build next to it)
    unless it is up to date; returns its path."""
    obj_dir, lib = (OBJ_CHECK, LIB_CHECK) if check else (OBJ, LIB)
    flags = NVCC_FLAGS + (["-DSZ3G_CHECK=1"] if check else [])
    stamp = _stamp() + ("-check" if check else "")
    stamp_file = os.path.join(obj_dir, "stamp")
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read() == stamp:
                return lib
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
