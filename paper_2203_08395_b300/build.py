"""Builds the CUDA library libhf.so (sm_103a) in-tree with nvcc.

Sources: csrc/api.cpp (C ABI, host graph builder), csrc/plan.cu (plans, executors, kernels),
csrc/costmodel.cu (learned cost model) and csrc/noalloc.cu (the allocation-free entry point).
The CUDA runtime is linked as a shared library so that, inside a process that already loaded
PyTorch's libcudart.so.13, both use one runtime instance.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libhf.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cpp", "plan.cu", "costmodel.cu", "noalloc.cu"]
HEADERS = ["hf_internal.h", "kernels.cuh", "team.cuh"]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "hf.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, ptxas_v=False):
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2,-Wall",
           "-shared", "-cudart", "shared", "-I", INCLUDE, "-o", tmp,
           *[os.path.join(CSRC, f) for f in SOURCES],
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    if ptxas_v:
        cmd.insert(1, "-Xptxas=-v")
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv)
    print(LIB)
