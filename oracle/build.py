"""Builds liboracle.so, the plain CPU FP64 reference (test infrastructure).

gcc only: -O2 -ffp-contract=off keeps every multiply and add separately
rounded in source order; OpenMP parallelises the outer spatial loop, which
does not change any result because every cell is computed independently.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
HDR = os.path.join(HERE, "oracle.h")
LIB = os.path.join(HERE, "liboracle.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in (SRC, HDR, __file__))


def build(force=False):
    """Compiles oracle.c into liboracle.so (if missing or stale); returns its path."""
    if not force and not _stale():
        return LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
            "-fPIC", "-shared", "-Wall", "-o", LIB + ".tmp", SRC]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        # no libgomp: the pragmas are ignored and the oracle runs on one thread
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
