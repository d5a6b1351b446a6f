"""Build libideq.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_2605_19705_gb300/libideq.so.  Host code is plain C++17; no architecture-
specific host flags are used, so the same command builds on x86_64 and aarch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libideq.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "net.cu", "kernels_elem.cu", "conv_simt.cu", "conv_tc.cu", "conv_edge.cu",
           "conv_edge_rb.cu", "fft.cu", "wgrad.cu",
           "net_train.cu", "noalloc.cu", "instr.cu", "wgrad_tc.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(debug: bool):
    f = ARCH + ["-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "--expt-relaxed-constexpr",
                "-I", os.path.join(HERE, "..", "include")]
    f += ["-O0", "-G"] if debug else ["-O3"]
    return f


def _compile(src: str, debug: bool, verbose_ptxas: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(debug)
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    for fn in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, fn)) > t:
            return True
    hdr = os.path.join(HERE, "..", "include", "ideq.h")
    return os.path.getmtime(hdr) > t or os.path.getmtime(__file__) > t


def build(force: bool = False, debug: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile and link libideq.so; returns its path."""
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, debug, verbose_ptxas), SOURCES))
    tmp = OUT + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, debug="--debug" in sys.argv,
          verbose_ptxas="-v" in sys.argv)
    print(OUT)
