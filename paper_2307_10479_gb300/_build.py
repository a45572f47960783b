"""Build libdeg.so in-tree with nvcc for sm_103a (GB300). Translation units compile in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdeg.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr"]
SOURCES = ["capi.cu", "search.cu", "search_f32.cu", "search_bf16.cu", "search_fp8.cu", "entry.cu", "layout.cu", "quantize.cu", "knn_exact.cu", "knn_tc.cu", "mlp.cu", "build_gpu.cu", "builder.cpp"]


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(HERE, "..", "include", "deg.h"))
    return hdrs


def _compile(src: str, extra: list[str]) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(OUT_DIR, src + ".o")
    newest = max(os.path.getmtime(p) for p in [path] + _deps())
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    if src.endswith(".cpp"):
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-c", path, "-o", obj]
    else:
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", path, "-o", obj]
    subprocess.run(cmd, check=True)
    return obj


def build(extra: list[str] | None = None, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libdeg.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = list(extra or [])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"],
                       check=True)
        os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
