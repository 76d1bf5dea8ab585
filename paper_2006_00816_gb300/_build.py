"""Build libhog.so from csrc/*.cu with nvcc for sm_103a (in-tree).

Each translation unit is compiled in parallel into ``_build/`` and linked
into ``paper_2006_00816_gb300/libhog.so``.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhog.so")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhog")


def _flags(verbose: bool):
    # host code: no floating-point contraction, so it rounds alike on x86-64
    # and aarch64 hosts
    f = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC] + ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    # diagnostic knob: extra nvcc flags for experimental builds (e.g. -DHOG_CORR_MINB=4)
    f += os.environ.get("HOG_NVCC_FLAGS", "").split()
    return f


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hm = _headers_mtime()
    cmd0 = [nvcc(), "-c"] + _flags(verbose)
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(OUT, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or verbose or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hm):
            jobs.append((s, o))
    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = {ex.submit(subprocess.run, cmd0 + [s, "-o", o], capture_output=True, text=True): s
                    for s, o in jobs}
            for fu in cf.as_completed(futs):
                r = fu.result()
                logs.append((futs[fu], r.stdout + r.stderr))
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed on %s:\n%s" % (futs[fu], r.stdout + r.stderr))
    if jobs or not os.path.exists(LIB) or force:
        tmp = LIB + ".tmp%d" % os.getpid()
        r = subprocess.run([nvcc(), "-shared"] + ARCH + ["-o", tmp] + objs + ["-lcudart", "-lpthread"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    if verbose:
        for s, txt in logs:
            print("==", os.path.basename(s))
            print(txt)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
