"""In-tree build of libto.so for sm_103a (GB300) with nvcc.

Each translation unit under ``csrc/`` compiles in parallel to an object file;
the objects link into ``_lib/libto.so``.  Rebuilds only when a source or
header is newer than the library.  ``build(checked=True)`` builds the
bounds-checked library instead (``-DTO_CHECKED``, objects in ``_lib/obj_checked``,
``_lib/libto_checked.so``; see ``toget_bounds_report`` in include/to.h).
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
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
SO = os.path.join(LIBDIR, "libto.so")
OBJDIR_CHECKED = os.path.join(LIBDIR, "obj_checked")
SO_CHECKED = os.path.join(LIBDIR, "libto_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libto.so")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "to.h"), __file__]


def stale(checked: bool = False) -> bool:
    so = SO_CHECKED if checked else SO
    if not os.path.exists(so):
        return True
    t = os.path.getmtime(so)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    so, objdir = (SO_CHECKED, OBJDIR_CHECKED) if checked else (SO, OBJDIR)
    if not force and not stale(checked):
        return so
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, "--expt-relaxed-constexpr"] + (["-DTO_CHECKED"] if checked else []) + list(extra_flags)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [cc, "-c", src, "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = so + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart=static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
