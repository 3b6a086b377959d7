"""Build ``libmf.so`` (the C-ABI library) from ``csrc/*.cu`` for sm_103a with nvcc.

Every translation unit is compiled in parallel, then linked with the static CUDA runtime.  The
result is written next to this file; build products go to ``_build/`` under the repository root.
``--debug`` builds the bounds-checked library ``libmf_debug.so`` instead (``-DMF_DEBUG_BOUNDS``:
index checks that record failures in a status word read by ``mf_debug_status``; objects in
``_build_debug/``).  Usage: ``python -m paper_2308_09839_gb300.build [--verbose-ptxas] [--debug]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libmf.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


DEBUG_LIB = os.path.join(PKG, "libmf_debug.so")


def _compile(src: str, ptxas_verbose: bool, debug: bool = False) -> tuple[str, str]:
    obj = os.path.join(BUILD + ("_debug" if debug else ""), os.path.basename(src).replace(".cu", ".o"))
    cmd = [nvcc(), *ARCH, *FLAGS, *(["-DMF_DEBUG_BOUNDS"] if debug else []), "-c", src, "-o", obj]
    if ptxas_verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj, r.stderr


def build(ptxas_verbose: bool = False, quiet: bool = True, debug: bool = False) -> str:
    out = DEBUG_LIB if debug else LIB
    os.makedirs(BUILD + ("_debug" if debug else ""), exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, ptxas_verbose, debug), srcs))
    objs = [o for o, _ in results]
    tmp = out + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, out)
    if not quiet or ptxas_verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    return out


if __name__ == "__main__":
    print(build(ptxas_verbose="--verbose-ptxas" in sys.argv, quiet=False, debug="--debug" in sys.argv))
