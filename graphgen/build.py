"""Compiles graphgen.c into libgraphgen.so beside this file (gcc, OpenMP when available), and
graphgen_dev.cu into libgraphgen_dev.so (nvcc, sm_103a; it calls libgraphgen.so for the host
part of the generator)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "graphgen.c")
HDR = os.path.join(HERE, "graphgen.h")
LIB = os.path.join(HERE, "libgraphgen.so")
DEV_SRC = os.path.join(HERE, "graphgen_dev.cu")
DEV_LIB = os.path.join(HERE, "libgraphgen_dev.so")


def _stale(lib, srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s) for s in srcs)


def needs_build() -> bool:
    return _stale(LIB, [SRC, HDR])


def command(openmp: bool = True):
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall", "-Wno-unused-function"]
    if openmp:
        cmd.append("-fopenmp")
    return cmd + [SRC, "-o", LIB]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def dev_command():
    return [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared", "-Xcompiler",
            "-fPIC", "-cudart", "static", "-I", HERE, DEV_SRC, "-o", DEV_LIB, "-L", HERE, "-lgraphgen",
            "-Xlinker", "-rpath,$ORIGIN"]


def build_dev(force: bool = False) -> str:
    """The device form (needs nvcc); returns its path."""
    build(force=False)
    if force or _stale(DEV_LIB, [DEV_SRC, HDR, LIB]):
        r = subprocess.run(dev_command(), capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("graphgen device build failed:\n" + r.stderr)
    return DEV_LIB


def build(force: bool = False) -> str:
    if force or needs_build():
        r = subprocess.run(command(True), capture_output=True, text=True)
        if r.returncode != 0:  # no libgomp: single-threaded build, same output
            r2 = subprocess.run(command(False), capture_output=True, text=True)
            if r2.returncode != 0:
                raise RuntimeError("graphgen build failed:\n" + r.stderr + r2.stderr)
    return LIB


def build_all(force: bool = False) -> None:
    build(force)
    build_dev(force)


if __name__ == "__main__":
    build_all(force=True)
    print(LIB, DEV_LIB)
