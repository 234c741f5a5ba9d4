"""Build libgamer_hydro.so in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked with
``nvcc -shared``.  Per-file flags:

* sweep_f32.cu: fast single-precision division / square root, FTZ
  (the FP32 path states its tolerance against the FP64 oracle);
* sweep_f64.cu, aux_kernels.cu: ``-fmad=false`` so FP64 results round
  exactly as the plain definition of the scheme;
* hydro_api.cu: host code of the C ABI;
* noalloc.cu: the allocation-free diagnostics entry point;
* regrid.cu: flag step and refinement fill of the refinement-map rebuild,
  ``-fmad=false`` (criteria in their plain order);
* poisson.cu: red-black SOR Poisson solver of one patch group per block,
  ``-fmad=false`` (FP64 in the oracle's order);
* gravity.cu: the gravity operator of the xyzGGzyx splitting,
  ``-fmad=false`` (FP64 in the oracle's order).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgamer_hydro.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", os.path.join(ROOT, "include"), "-I", CSRC]
UNITS = {
    "sweep_f32.cu": ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "sweep_f64.cu": ["-fmad=false"],
    "aux_kernels.cu": ["-fmad=false"],
    "hydro_api.cu": [],
    "noalloc.cu": [],
    "regrid.cu": ["-fmad=false"],
    "poisson.cu": ["-fmad=false"],
    "gravity.cu": ["-fmad=false"],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "gamer_hydro.h"))
    files.append(os.path.abspath(__file__))
    return any(os.path.getmtime(f) > t for f in files)


def build(force: bool = False, verbose: bool = False, extra=None) -> str:
    """Compile and link; returns the path of the shared library."""
    if not force and not _sources_newer_than(LIB):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    extra = list(extra or [])

    def one(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(OUT_DIR, name.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *UNITS[name], *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(one, UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force=True, verbose=v, extra=["-Xptxas", "-v"] if v else None))
