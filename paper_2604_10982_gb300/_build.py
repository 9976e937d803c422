"""Build libpsi.so in-tree for sm_103a with nvcc (translation units compiled in
parallel, then linked with the static CUDA runtime)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpsi.so")
# the same sources compiled with PSI_DEBUG: bounds checks of the indices the
# pipeline kernels take from data (see psi_debug_checks in psi.h)
OUT_DEBUG = os.path.join(OUT, "debug")
LIB_DEBUG = os.path.join(OUT, "libpsi_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "project.cu", "intersect.cu", "sort.cu", "render_fwd.cu", "render_bwd.cu", "feat_bwd.cu",
           "decode.cu", "labels.cu", "regularisers.cu", "frames.cu", "attention.cu", "geometry.cu", "quantize.cu", "fill.cu"]
# the binning path takes integer decisions in float32 with an explicit
# operation order: forbid FMA contraction there as well
NO_FMAD = {"project.cu", "intersect.cu"}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _deps():
    return glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "psi.h")]


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, debug: bool = False) -> str:
    """Build libpsi.so (or, with debug, libpsi_debug.so) if a source changed."""
    lib, out = (LIB_DEBUG, OUT_DEBUG) if debug else (LIB, OUT)
    if not force and not needs_build(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
                     "--expt-relaxed-constexpr"] + (["-DPSI_DEBUG"] if debug else [])
    if ptxas_v:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [nvcc] + common + (["-fmad=false"] if src in NO_FMAD else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or (ptxas_v and r.stderr):
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> None:
    """The release and the debug library, their translation units compiled in parallel."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        list(ex.map(lambda d: build(force=force, debug=d), (False, True)))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
