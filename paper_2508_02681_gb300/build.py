"""In-tree build of the CUDA library ``libunocg.so`` for sm_103a (no CMake, parallel nvcc)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.environ.get("UNOCG_BUILD_DIR", os.path.join(ROOT, "_build"))
LIB = os.environ.get("UNOCG_LIB_OUT", os.path.join(HERE, "libunocg.so"))
SOURCES = ["api.cu", "k_stencil.cu", "k_setup.cu", "k_fft_plane.cu", "k_line64.cu", "k_line32.cu", "k_persist.cu",
           "k_fft_reg.cu", "k_ku_tma.cu", "k_ku_vec.cu", "k_ku_el2.cu", "k_newton.cu", "k_line_tma.cu", "k_line_tma3.cu", "k_line_tp.cu", "k_plane_cl.cu", "dirichlet/k_dirichlet.cu", "dirichlet/k_dirichlet_reg.cu", "dirichlet/api_dirichlet.cu"]
# loads of data written by other blocks of the same launch must bypass L1
PER_FILE = {"k_persist.cu": ["-Xptxas", "-dlcm=cg"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src: str, extra) -> str:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0].replace("/", "_") + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *PER_FILE.get(src, []), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False, extra=()) -> str:
    """Compile every translation unit (in parallel) and link ``libunocg.so`` in the package."""
    os.makedirs(OUT_DIR, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra)), SOURCES))
    cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
