"""Build liblsgpu.so in-tree: CUDA kernels for sm_103a plus the host setup.

    python paper_2608_17615_b300/build.py
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "liblsgpu.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _run(cmd):
    print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)


def build(verbose_ptxas=False):
    os.makedirs(BUILD, exist_ok=True)
    cu_obj = os.path.join(BUILD, "lsgpu.o")
    cpp_obj = os.path.join(BUILD, "setup.o")
    nv = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp",
          "-c", os.path.join(CSRC, "lsgpu.cu"), "-o", cu_obj]
    if verbose_ptxas:
        nv.insert(1, "-Xptxas=-v")
    _run(nv)
    _run(["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", "-c", os.path.join(CSRC, "setup.cpp"), "-o", cpp_obj])
    _run([NVCC, "-shared", *ARCH, "-o", LIB, cu_obj, cpp_obj, "-lcusolver", "-lcublas", "-Xcompiler", "-fopenmp"])
    return LIB


if __name__ == "__main__":
    build(verbose_ptxas="-v" in sys.argv)
