"""Build libptn.so in-tree for sm_103a (nvcc + g++, objects compiled in parallel).

Usage: python -m paper_2604_08467_gb300.build_lib [--force]
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libptn.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ffp-contract=off keeps host FP64 table arithmetic (Kraus probabilities and
# CDFs) free of fused multiply-adds, so it rounds like the specification.
HOST_FLAGS = ["-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-Wall", "-Wno-unused-function"]
CU_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler",
            "-fPIC,-ffp-contract=off", "-I" + INCLUDE] + ARCH

CPP_SOURCES = ["planner.cpp"]
CU_SOURCES = ["runtime.cu", "kernels_contract.cu", "kernels_sample.cu", "kernels_gemm.cu", "stats.cu", "noalloc.cu",
              "kernels_expval.cu", "kernels_merge.cu", "kernels_harvest.cu", "tune.cu",
              "kernels_cache.cu"]


def _sources():
    return [os.path.join(CSRC, f) for f in CPP_SOURCES + CU_SOURCES]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = _sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(INCLUDE, "ptn.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    if src.endswith(".cpp"):
        cmd = [NVCC, "-x", "c++", "-c", src, "-o", obj, "-I" + INCLUDE, "-Xcompiler",
               ",".join(HOST_FLAGS)]
    else:
        cmd = [NVCC, "-c", src, "-o", obj] + CU_FLAGS
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force=False, verbose=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and not _stale():
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(_sources())) as ex:
        results = list(ex.map(_compile, _sources()))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log.strip():
                print(log)
    tmp = LIB + ".tmp"
    cmd = [NVCC, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
