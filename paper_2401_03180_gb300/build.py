"""Compile the CUDA library (libmdgb.so) in-tree for sm_103a.

nvcc compiles each translation unit in parallel and links one shared
library with a C ABI (include/md.h).  Host code is built without
floating-point contraction, and the charge-update kernels without FMA
(-fmad=false), because those results must match a CPU reference bit for bit.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmdgb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = {
    "md_host.cu": [],
    "k_step.cu": ["-fmad=false"],
    "k_cells.cu": [],
    "k_pair.cu": [],
    "md_noalloc.cu": [],
    "k_probe.cu": ["-fmad=false"],
    "k_frag.cu": [],
    "k_peak.cu": [],
}


def _nvcc() -> str:
    cand = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"), "nvcc"]
    for c in cand:
        if shutil.which(c) or os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmdgb.so")


def _common(extra_ptxas: bool) -> list[str]:
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
             "--expt-relaxed-constexpr", f"-I{os.path.join(ROOT, 'include')}", *ARCH]
    if extra_ptxas:
        flags += ["-Xptxas", "-v"]
    return flags


def _digest(paths) -> str:
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode() + f.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "md.h"))
    deps.append(os.path.abspath(__file__))
    stamp = os.path.join(BUILD, "stamp")
    dg = _digest(deps)

    def current():
        return os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == dg

    if not force and current():
        return LIB
    # one builder at a time (several ranks of one job may call this at once);
    # the others find the library current once they hold the lock
    import fcntl
    with open(os.path.join(BUILD, "lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            if not force and current():
                return LIB
            return _compile(dg, stamp, verbose, ptxas_info)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _compile(dg: str, stamp: str, verbose: bool, ptxas_info: bool) -> str:
    nvcc = _nvcc()

    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, *_common(ptxas_info), *SOURCES[src]]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(one, SOURCES))
    if verbose or ptxas_info:
        for obj, log in results:
            if log.strip():
                print(f"--- {os.path.basename(obj)}\n{log}")
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, "-shared", "-o", tmp, *[o for o, _ in results], *ARCH, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dg)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
