"""Compile the oracle's C sources into oracle/liboracle.so (gcc, OpenMP).

Test infrastructure only: nothing on the library's compute path uses it."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, "sv.c"), os.path.join(HERE, "sector.c")]


def build(force: bool = False) -> str:
    if not force and os.path.exists(SO) and all(
            os.path.getmtime(SO) >= os.path.getmtime(s) for s in SRC):
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp] + SRC + ["-lm"])
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True))
