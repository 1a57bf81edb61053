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
    """Compile every csrc/*.cu with nvcc (sm_103a) and csrc/*.cpp with g++, link liblsgpu.so."""
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    for name in sorted(os.listdir(CSRC)):
        src = os.path.join(CSRC, name)
        obj = os.path.join(BUILD, os.path.splitext(name)[0] + ".o")
        if name.endswith(".cu"):
            nv = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp", "-c", src, "-o", obj]
            if verbose_ptxas:
                nv.insert(1, "-Xptxas=-v")
            _run(nv)
        elif name.endswith(".cpp"):
            _run(["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", "-c", src, "-o", obj])
        else:
            continue
        objs.append(obj)
    _run([NVCC, "-shared", *ARCH, "-o", LIB, *objs, "-lcusolver", "-lcublas", "-lcufft", "-Xcompiler", "-fopenmp"])
    return LIB


if __name__ == "__main__":
    build(verbose_ptxas="-v" in sys.argv)
