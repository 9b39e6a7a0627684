"""Compiles oracle.c into liboracle.so beside this file (plain gcc, single-threaded)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def needs_build() -> bool:
    return not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC)


def command():
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", SRC, "-o", LIB]


def build(force: bool = False) -> str:
    if force or needs_build():
        r = subprocess.run(command(), capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
