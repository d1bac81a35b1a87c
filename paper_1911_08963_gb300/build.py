"""Build the CUDA library libmd.so in-tree (nvcc, sm_103a only).

    python -m paper_1911_08963_gb300.build            # libmd.so
    python -m paper_1911_08963_gb300.build --debug    # libmd_debug.so, range checks on (-DMD_DEBUG_BOUNDS)
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libmd.so")
DEBUG_OBJDIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(LIBDIR, "libmd_debug.so")
SOURCES = ["md_kernels.cu", "md_engine.cu", "md_host.cpp", "md_capi.cpp", "md_engine.cpp", "md_server.cpp", "md_noalloc.cu",
           "md_tc.cu", "md_tune.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
# extra nvcc flags for tuning experiments (e.g. -DMD_UPPERS_PER_LANE=4); empty by default
COMMON += os.environ.get("MD_NVCC_FLAGS", "").split()


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return out + [os.path.join(INCLUDE, "md.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile what is stale, under a file lock (several ranks may call this at once).
    debug: the range-checked library (libmd_debug.so), built from the same sources."""
    import fcntl
    os.makedirs(DEBUG_OBJDIR if debug else OBJDIR, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    with open(os.path.join(LIBDIR, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(force, verbose, debug)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(force: bool, verbose: bool, debug: bool = False) -> str:
    objdir = DEBUG_OBJDIR if debug else OBJDIR
    lib = DEBUG_LIB if debug else LIB
    flags = COMMON + (["-DMD_DEBUG_BOUNDS"] if debug else [])
    cc = nvcc()
    headers = _deps()
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    objs = []
    jobs = []
    for s in srcs:
        src = os.path.join(CSRC, s)
        obj = os.path.join(objdir, s + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [cc] + ARCH + flags + ["-c", src, "-o", obj]
            if s.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
