"""Build the CUDA library ``libgals.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` file is compiled by nvcc in parallel into ``_build/*.o`` and the
objects are linked into ``paper_0905_3409_gb300/libgals.so``.  Only the files whose
sources (or the shared headers) changed are recompiled.

A stamp in each build directory records the machine, the nvcc version and the flags; a
build whose stamp differs starts from no objects (``clean=True`` forces that).

``build_checked()`` builds the same sources with ``-DGALS_CHECKED`` into
``libgals_checked.so`` (objects in ``_build_checked``): the step kernels test their
data-dependent indexes and report a violation through the grid's error word.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libgals.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgals.so")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(ROOT, "include", "gals.h")]


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _stamp_text(extra) -> str:
    """What the objects of a build directory depend on besides their sources: the host
    (objects of another machine are never reused), the compiler and every flag."""
    try:
        ver = subprocess.run([nvcc(), "--version"], capture_output=True, text=True).stdout.strip().splitlines()[-1]
    except (OSError, IndexError):
        ver = "unknown"
    return "\n".join([platform.machine(), ver] + ARCH + NVCC_FLAGS + list(extra)) + "\n"


def _check_stamp(build_dir: str, extra, clean: bool) -> None:
    """Empty the build directory when asked to, or when its stamp (machine, nvcc, flags)
    differs from this build's; then write the stamp."""
    stamp = os.path.join(build_dir, "STAMP")
    want = _stamp_text(extra)
    have = open(stamp).read() if os.path.exists(stamp) else None
    if clean or have != want:
        for fn in glob.glob(os.path.join(build_dir, "*.o")):
            os.remove(fn)
    with open(stamp, "w") as f:
        f.write(want)


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra=(), build_dir: str = BUILD, lib: str = LIB, clean: bool = False) -> str:
    """Compile what changed (every object when `clean`, or when the machine, the compiler
    or the flags differ from the last build in build_dir) and link the library."""
    os.makedirs(build_dir, exist_ok=True)
    _check_stamp(build_dir, extra, clean)
    if clean and os.path.exists(lib):
        os.remove(lib)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    if _stale(lib, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", lib + ".tmp"] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(lib + ".tmp", lib)
    if verbose:
        print(f"built {lib}")
    return lib


def build_checked(verbose: bool = False, clean: bool = False) -> str:
    """The checked build: libgals_checked.so (see the module docstring)."""
    return build(verbose, extra=("-DGALS_CHECKED",), build_dir=os.path.join(HERE, "_build_checked"),
                 lib=os.path.join(HERE, "libgals_checked.so"), clean=clean)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if a != "--clean"]
    build(verbose=True, extra=args, clean="--clean" in sys.argv[1:])
