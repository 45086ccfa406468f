"""Build the CE CUDA library in-tree: ``paper_1603_09133_gb300/libcegpu.so``.

Every translation unit is compiled for sm_103a only, in parallel, then linked
with the shared CUDA runtime (so device pointers and streams from PyTorch are
used directly).  ``python -m paper_1603_09133_gb300.build`` runs it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcegpu.so")
SOURCES = ["api.cu", "row_kernel.cu", "factor_kernels.cu", "apply_kernels.cu", "pcg_noalloc.cu", "pcg_batched.cu", "minres.cu",
           "mlp.cu", "probes.cu", "big_rows.cu", "tc_gemm.cu", "plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CE library needs the CUDA toolkit")
    return cand


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
           "-I", os.path.join(HERE, "..", "include"), *ARCH, "-c",
           os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd.insert(1, "--expt-relaxed-constexpr")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    if verbose:
        sys.stderr.write(res.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "ce.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link ``libcegpu.so`` (skipped when it is up to date)."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + ".tmp"
    cudalib = os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "lib64")
    cmd = [_nvcc(), "-shared", *ARCH, "-cudart", "shared",
           "-Xlinker", f"-rpath={cudalib}", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
