"""Build libpmlbie.so in-tree for sm_103a (nvcc + g++, no cmake).

Usage: python -m paper_2412_11162_gb300.build  (or call build()).
"""
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libpmlbie.so")
BUILD = os.path.join(HERE, "_build")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", "-I" + os.path.join(CUDA, "include")]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stderr


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    srcs_cu = ["kernels.cu", "kernels_ff.cu", "lu.cu", "gmres.cu", "api.cu", "noalloc.cu", "probe.cu"]
    srcs_cc = ["host.cpp"]
    jobs = []
    for s in srcs_cu:
        jobs.append([NVCC, "-c", os.path.join(CSRC, s), "-o", os.path.join(BUILD, s + ".o")] + CU_FLAGS)
    for s in srcs_cc:
        jobs.append(["g++", "-c", os.path.join(CSRC, s), "-o", os.path.join(BUILD, s + ".o")] + CXX_FLAGS)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    objs = [os.path.join(BUILD, s + ".o") for s in srcs_cu + srcs_cc]
    extra = ["-lquadmath"] if platform.machine() in ("x86_64", "AMD64") else []
    _run([NVCC, "-shared", "-o", OUT] + objs + ARCH + ["-lcudart", "-lpthread"] + extra)
    if verbose:
        for l in logs:
            sys.stderr.write(l)
    return OUT


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
    print(OUT)
