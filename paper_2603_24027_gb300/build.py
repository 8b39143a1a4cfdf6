"""Build libfdtd_gb300.so (sm_103a) in-tree with nvcc.

Each .cu translation unit compiles in parallel to an object under _build/,
then nvcc links the shared library next to this file.  Only one -gencode
target: the GB300 (compute_103a / sm_103a).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "libfdtd_gb300.so")
# Bounds-checked variant for tests (-DFDTD_BOUNDS_CHECK): every store of the
# default kernels checks that it lands in a buffer the launch may write.
LIB_CHECKED = os.path.join(HERE, "libfdtd_gb300_checked.so")
SOURCES = ["kernels_step.cu", "kernels_lag2.cu", "kernels_rev_fused.cu", "kernels_fwd_fused.cu",
           "kernels_fwd_2step.cu", "tensor_maps.cu", "kernels_tape.cu", "kernels_bdct.cu", "fdtd_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + INCLUDE]


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(home, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "fdtd.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()[:16]


# Device code of the default half-step kernels: the files whose change can
# change what those kernels move through memory.
KERNEL_FILES = ["kernels_lag2.cu", "kernels_rev_fused.cu", "kernels_fwd_fused.cu",
                "kernels_fwd_2step.cu", "lag_common.cuh", "fdtd_internal.cuh", "tma.cuh"]


def kernel_digest() -> str:
    """Digest of the default kernels' device code and compile flags (keys the
    recorded DRAM traffic per launch: host-only changes keep it valid).  The
    include path is left out, so that copies of the tree at other paths (and
    machines) agree."""
    h = hashlib.sha256()
    for name in KERNEL_FILES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    h.update(" ".join(ARCH + [x for x in FLAGS if not x.startswith("-I")]).encode())
    return h.hexdigest()[:16]


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    out = LIB_CHECKED if checked else LIB
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    extra = list(extra) + (["-DFDTD_BOUNDS_CHECK"] if checked else [])
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, "libfdtd_gb300.stamp")
    dig = _digest()
    if not force and os.path.exists(out) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return out

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    with open(stamp, "w") as f:
        f.write(dig)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ()))
