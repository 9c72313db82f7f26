"""Build the engine in-tree: paper_2510_15413_b300/libfhesql.so for sm_103a.

host.cpp (key generation, encryption, circuit scheduler) is compiled by g++
without fast-math or floating-point contraction, so the Gaussian sampler is
the host libm's; kernels.cu by nvcc for sm_103a only.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfhesql.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["host.cpp", "kernels.cu", "server.cu", "plain.cu", "peaks.cu", "schedule.cu", "engine.h", "ntt.cuh",
           "br_split.cuh"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(ROOT, "include", "fhesql.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include")]
    host_o = os.path.join(BUILD, "host.o")
    dev_o = os.path.join(BUILD, "kernels.o")
    srv_o = os.path.join(BUILD, "server.o")
    lit_o = os.path.join(BUILD, "plain.o")
    pk_o = os.path.join(BUILD, "peaks.o")
    sc_o = os.path.join(BUILD, "schedule.o")
    run = lambda cmd: subprocess.run(cmd, check=True, capture_output=not verbose)
    run(["g++", "-std=c++17", "-O2", "-fPIC", "-fvisibility=hidden", "-fno-fast-math", "-ffp-contract=off",
         "-pthread", "-Wall", "-Wextra", *inc, "-c", os.path.join(CSRC, "host.cpp"), "-o", host_o])
    run([NVCC, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xptxas", "-v", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         *inc, "-c", os.path.join(CSRC, "kernels.cu"), "-o", dev_o])
    run([NVCC, "-std=c++17", "-O2", *ARCH, "-Xcompiler", "-fPIC,-fvisibility=hidden,-pthread",
         *inc, "-c", os.path.join(CSRC, "server.cu"), "-o", srv_o])
    run([NVCC, "-std=c++17", "-O2", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         *inc, "-c", os.path.join(CSRC, "plain.cu"), "-o", lit_o])
    run([NVCC, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         *inc, "-c", os.path.join(CSRC, "peaks.cu"), "-o", pk_o])
    run([NVCC, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         *inc, "-c", os.path.join(CSRC, "schedule.cu"), "-o", sc_o])
    tmp = LIB + f".tmp{os.getpid()}"
    run([NVCC, "-shared", *ARCH, host_o, dev_o, srv_o, lit_o, pk_o, sc_o, "-o", tmp, "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
