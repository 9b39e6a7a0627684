"""Compiles graphgen.c into libgraphgen.so beside this file (gcc, OpenMP when available)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "graphgen.c")
LIB = os.path.join(HERE, "libgraphgen.so")


def needs_build() -> bool:
    return not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC)


def command(openmp: bool = True):
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall", "-Wno-unused-function"]
    if openmp:
        cmd.append("-fopenmp")
    return cmd + [SRC, "-o", LIB]


def build(force: bool = False) -> str:
    if force or needs_build():
        r = subprocess.run(command(True), capture_output=True, text=True)
        if r.returncode != 0:  # no libgomp: single-threaded build, same output
            r2 = subprocess.run(command(False), capture_output=True, text=True)
            if r2.returncode != 0:
                raise RuntimeError("graphgen build failed:\n" + r.stderr + r2.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
