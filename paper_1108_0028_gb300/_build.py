"""Compile the CUDA sources of the library into ``paper_1108_0028_gb300/librcb.so`` (sm_103a).

Each ``csrc/*.cu`` is compiled to an object in ``_build/`` (in parallel), then linked with
``nvcc -shared``.  Objects are rebuilt when their source or any header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librcb.so")
PEAK_SRC = os.path.join(HERE, "peak", "alu_rate.cu")
PEAK_LIB = os.path.join(HERE, "libpeak.so")  # arithmetic-rate probe of the benchmark (not part of the C ABI)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
# float32-heavy kernels: flush subnormals and use the hardware reciprocal / square-root
# approximations (the walk and neighbour filters carry an absolute slack of 1e-30 for this;
# float64 arithmetic is unaffected)
FAST_FP32 = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
FAST_FILES = {"gravity.cu", "neighbours.cu", "walk.cu"}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    newest_header = max([os.path.getmtime(h) for h in headers] + [os.path.getmtime(__file__)])
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_header):
            return obj, ""
        cmd = [nvcc] + ARCH + FLAGS + (FAST_FP32 if os.path.basename(src) in FAST_FILES else []) + \
            ["-c", src, "-o", obj + ".tmp"]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose:
        for o, log in results:
            if log:
                print(f"== {os.path.basename(o)}\n{log}")
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    if force or not os.path.exists(PEAK_LIB) or os.path.getmtime(PEAK_LIB) < os.path.getmtime(PEAK_SRC):
        cmd = [nvcc] + ARCH + ["-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "-o", PEAK_LIB + ".tmp", PEAK_SRC]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {PEAK_SRC}:\n{r.stderr}")
        os.replace(PEAK_LIB + ".tmp", PEAK_LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
