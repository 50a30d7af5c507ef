"""Build the CUDA library libns_adjoint.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel to an object file, then linked into one
shared library next to this file.  Run as ``python -m paper_1511_06959_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libns_adjoint.so")
BUILD = os.path.join(HERE, "_build")
# bounds-checking build: every field access of the stencil kernels is checked against its
# field's extent (NS_DEBUG_BOUNDS, NS_ERR_BOUNDS in the sticky error word); load it with
# NS_ADJOINT_LIB=<OUT_DEBUG>
OUT_DEBUG = os.path.join(HERE, "libns_adjoint_debug.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
SOURCES = ["ns_rhs.cu", "ns_adj.cu", "ns_diag.cu", "ns_api.cu", "ns_sweep.cu", "ns_noalloc.cu", "ns_mlp.cu",
           "ns_lambda.cu", "ns_probe.cu", "ns_bc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Single-precision division and square root in the fast form (-prec-div/-prec-sqrt off):
# a few units in the last place instead of correctly rounded, in the FP32 products of the
# mixed path only (FP64 is unaffected); the stencil and sigma_1 kernels spend many of
# their instructions on them.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills", "-prec-div=false", "-prec-sqrt=false"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return exe


def _compile(src: str, extra, bdir: str = BUILD) -> str:
    obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip():
        sys.stderr.write(r.stderr)
    return obj


def build(verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile and link the library; debug: the bounds-checking build (OUT_DEBUG)."""
    bdir, out = (BUILD_DEBUG, OUT_DEBUG) if debug else (BUILD, OUT)
    os.makedirs(bdir, exist_ok=True)
    flags = list(extra) + (["-DNS_DEBUG_BOUNDS"] if debug else [])
    if verbose:
        flags += ["-Xptxas", "-v"]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags, bdir), SOURCES))
    cmd = [nvcc(), *ARCH, "-shared", "-o", out, *objs, "-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug="--debug" in sys.argv))
