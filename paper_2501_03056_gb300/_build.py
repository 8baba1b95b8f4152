"""Build of the CUDA library ``_lib/libfppg.so`` for GB300 (sm_103a).

Each translation unit is compiled by nvcc in parallel and linked into one
shared library with the CUDA runtime linked statically.  ``mesh.cu`` (the
FP64 set-up) is compiled without FMA contraction so that its feature and
normal arithmetic is evaluated exactly in the written order; the host parts
of ``mapping.cu`` and ``curve.cu`` (feature particles, intersection curve)
are compiled without contraction by the host compiler as well.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libfppg.so")
LIB_CHECKED = os.path.join(LIBDIR, "libfppg_checked.so")   # the bounds-checked build (-DFPPG_CHECKED)
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", os.path.join(ROOT, "include")]
UNITS = {
    "sort.cu": [],
    "mesh.cu": ["-fmad=false"],
    "body.cu": [],
    "relax.cu": [],
    "energy.cu": [],
    "api.cu": [],
    "noalloc.cu": [],
    "mapping.cu": ["-fmad=false", "-Xcompiler", "-ffp-contract=off"],
    "union.cu": ["-fmad=false"],
    "curve.cu": ["-fmad=false", "-Xcompiler", "-ffp-contract=off"],
    "intervals.cu": [],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the FPPG library needs the CUDA toolkit to build")
    return p


def _sources_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "fppg.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checked: bool = False) -> str:
    """Compile every unit and link the shared library; returns its path.
    checked: the bounds-checked build (every hot-path kernel checks the
    indices it computes, fppg_check_status reports failures), linked as a
    library of its own."""
    os.makedirs(LIBDIR, exist_ok=True)
    out = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _sources_mtime():
        return out
    cc = nvcc()
    objdir = os.path.join(LIBDIR, "obj_checked" if checked else "obj")
    os.makedirs(objdir, exist_ok=True)
    extra = list(extra or []) + (["-DFPPG_CHECKED"] if checked else [])

    def compile_one(item):
        src, flags = item
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS.items()))
    tmp = out + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", *objs, "-lpthread", "-ldl", "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
