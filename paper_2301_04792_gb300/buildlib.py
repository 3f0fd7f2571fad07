"""In-tree build of ``liblb.so`` (the C ABI declared in ``include/lb.h``).

Each ``csrc/*.cu`` translation unit is compiled by nvcc for sm_103a only, in
parallel, then linked into one shared library with the CUDA runtime linked
statically (so the library loads on a machine without a GPU; calls then fail
with LB_ERR_CUDA).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblb.so")
HEADER = os.path.join(ROOT, "include", "lb.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblb.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))) + [HEADER]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc(), "-c", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(ROOT, "include"), *extra, "-o", obj, src]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, extra_flags=(), verbose: bool = False) -> str:
    """Compile and link ``liblb.so`` if any source changed; returns its path."""
    with _lock:
        if not force and not stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        srcs = sources()
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            objs = list(ex.map(lambda s: _compile(s, list(extra_flags)), srcs))
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), "-shared", "-cudart", "static", *ARCH, "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        if verbose:
            print(f"built {LIB}")
        return LIB


def ptxas_report() -> str:
    """Registers / spills / shared memory of every kernel (nvcc -Xptxas -v)."""
    os.makedirs(BUILD, exist_ok=True)
    out = []
    for src in sources():
        cmd = [nvcc(), "-c", "-O3", "-std=c++17", *ARCH, "-Xptxas", "-v", "-Xcompiler", "-fPIC",
               "-I", os.path.join(ROOT, "include"), "-o", os.path.join(BUILD, "ptxas_probe.o"), src]
        r = subprocess.run(cmd, capture_output=True, text=True)
        out.append(r.stderr)
    return "\n".join(out)


if __name__ == "__main__":
    build(force=True, verbose=True)
