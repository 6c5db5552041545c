"""Builds liblbm.so (the CUDA library behind include/lbm.h) in-tree for sm_103a,
and its debug build liblbm_debug.so (LBM_DEBUG: every population access of
the kernels index-checked, a failed check recorded and skipped; see
include/lbm.h).

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into one shared library next to this file.  Rebuilds only when a source or
header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblbm.so")
OBJDIR = os.path.join(HERE, "_build")
DEBUG_LIB = os.path.join(HERE, "liblbm_debug.so")
DEBUG_OBJDIR = os.path.join(HERE, "_build", "debug")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++20", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"] + ARCH


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + [os.path.join(ROOT, "include", "lbm.h"), __file__]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _variants(debug: bool | None):
    """(library, object folder, extra nvcc flags) of the requested builds:
    release only (False), debug only (True) or both (None)."""
    v = []
    if debug is not True:
        v.append((LIB, OBJDIR, ()))
    if debug is not False:
        v.append((DEBUG_LIB, DEBUG_OBJDIR, ("-DLBM_DEBUG",)))
    return v


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          debug: bool | None = False) -> str:
    """Builds the release library (debug=False), the debug library
    (debug=True) or both in one parallel pass (debug=None); returns the path
    of the release library, or of the debug one when only it was asked for."""
    todo = [v for v in _variants(debug) if force or not up_to_date(v[0])]
    result = DEBUG_LIB if debug is True else LIB
    if not todo:
        return result
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(job):
        src, objdir, flags = job
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, *flags, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    jobs = []
    for _, objdir, flags in todo:
        os.makedirs(objdir, exist_ok=True)
        jobs += [(src, objdir, flags) for src in sources()]
    # the largest translation units first, so that they do not finish last
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        results = dict(zip(jobs, ex.map(compile_one, jobs)))
    if verbose or ptxas_info:
        for _, log in results.values():
            if log.strip():
                print(log)
    for lib, objdir, flags in todo:
        objs = [results[(src, objdir, flags)][0] for src in sources()]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return result


if __name__ == "__main__":
    import sys
    which = None if "--all" in sys.argv else ("--debug" in sys.argv)
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                debug=which))
