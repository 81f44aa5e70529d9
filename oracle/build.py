"""Compile the oracle's C primitives into oracle/_build/liboracle.so.

Test infrastructure: the CPU oracle is built here and loaded only by tests,
the smoke check and bench.py's CPU-baseline leg.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ckks_core.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Build the shared library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run(
        ["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC", SRC, "-o", tmp,
         "-lquadmath", "-lm"],
        check=True,
    )
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
