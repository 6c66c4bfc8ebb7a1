"""Build the CUDA library libgkogb.so in-tree with nvcc for sm_103a.

Every .cu under csrc/ is compiled to an object in parallel, then linked
into paper_2011_08879_gb300/libgkogb.so.  A second copy of the library,
libgkogb_checked.so, is compiled with -DGKO_CHECK_BOUNDS: its kernels clamp
indices that the caller did not validate and report them through the error
word (kErrBadIndex) instead of reading or writing out of range; the tests of
that failure path load it.  Objects are rebuilt only when a source or header
is newer.  Run ``python -m paper_2011_08879_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgkogb.so")
OBJDIR_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libgkogb_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "--extended-lambda", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose, checked=False):
    obj = os.path.join(OBJDIR_CHECKED if checked else OBJDIR, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + _headers()):
        return obj, ""
    cmd = [nvcc(), *ARCH, *FLAGS, *(["-DGKO_CHECK_BOUNDS"] if checked else []), "-I", INCLUDE, "-c", src, "-o",
           obj + ".tmp"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, p.stdout, p.stderr))
    os.replace(obj + ".tmp", obj)
    return obj, p.stderr


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link the library and its bounds-checked copy; returns the
    library's path."""
    os.makedirs(OBJDIR, exist_ok=True)
    os.makedirs(OBJDIR_CHECKED, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    todo = [(s, False) for s in srcs] + [(s, True) for s in srcs]
    jobs = jobs or min(len(todo), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda sc: _compile(sc[0], verbose, sc[1]), todo))
    if verbose:
        for _, log in results[:len(srcs)]:
            if log:
                sys.stderr.write(log)
    for lib, objs in ((LIB, [o for o, _ in results[:len(srcs)]]), (LIB_CHECKED, [o for o, _ in results[len(srcs):]])):
        if _stale(lib, objs):
            tmp = lib + ".tmp%d" % os.getpid()
            cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
            p = subprocess.run(cmd, capture_output=True, text=True)
            if p.returncode != 0:
                raise RuntimeError("link failed:\n%s\n%s" % (p.stdout, p.stderr))
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
