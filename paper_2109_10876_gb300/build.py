"""Compile the CUDA library (csrc/*.cu) for sm_103a into lib/libmd_gb300.so,
and its checked build (-DMD_CHECKED: device-side bounds checks that latch
MD_ERR_BOUNDS instead of trapping) into lib/libmd_gb300_checked.so.

Every translation unit of both builds is compiled by nvcc in parallel, then
each build is linked into one shared library with the CUDA runtime linked
statically.  The results are in-tree (paper_2109_10876_gb300/lib/) and
git-ignored.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libmd_gb300.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libmd_gb300_checked.so")
# build name -> (extra nvcc flags, object directory, library)
VARIANTS = {
    "default": ([], OUT_DIR, LIB),
    "checked": (["-DMD_CHECKED"], os.path.join(OUT_DIR, "checked"), LIB_CHECKED),
}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", INCLUDE, "-I", CSRC]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra_flags=(), variants=("default", "checked")):
    """Build the named variants; returns the default library's path."""
    srcs = _sources()
    hdrs = _headers()
    objs, jobs = {}, []
    for v in variants:
        vflags, odir, _ = VARIANTS[v]
        os.makedirs(odir, exist_ok=True)
        objs[v] = [os.path.join(odir, os.path.basename(s)[:-3] + ".o") for s in srcs]
        jobs += [(s, o, vflags) for s, o in zip(srcs, objs[v]) if force or _stale(o, [s] + hdrs)]
    cc = nvcc()

    def compile_one(job):
        s, o, vflags = job
        cmd = [cc, *ARCH, *NVCC_FLAGS, *vflags, *extra_flags, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr}")
        return r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for msg in ex.map(compile_one, jobs):
                if verbose and msg:
                    print(msg, file=sys.stderr)
    for v in variants:
        lib = VARIANTS[v][2]
        if force or _stale(lib, objs[v]):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs[v]]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.run(cmd, check=True)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    var = ("default",) if "--default-only" in sys.argv else ("default", "checked")
    print(build(force="--force" in sys.argv or bool(extra), verbose=v or bool(extra), extra_flags=extra,
                variants=var))
