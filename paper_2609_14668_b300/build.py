"""Build libafqmc.so in place with nvcc for sm_103a (B300)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libafqmc.so")
SOURCES = ["csrc/afqmc.cu"]
HEADERS = ["csrc/common.cuh", "csrc/learned.cuh", "csrc/linalg.cuh", "csrc/measure.cuh", "csrc/ozaki.cuh",
           "csrc/tdgf.cuh", "csrc/update.cuh", "csrc/wrap.cuh"]


def nvcc_command(out=LIB):
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    return [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
            "-Xcompiler", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "include"),
            "-o", out] + [os.path.join(HERE, s) for s in SOURCES]


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(HERE, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "afqmc.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    if not force and not stale():
        return LIB
    cmd = nvcc_command()
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
