"""Build the CPU oracle shared library (oracle/liboracle.so).

Test infrastructure: the oracle is only loaded by tests/, __graft_entry__.smoke()
and bench.py's CPU baseline / reference leg.  Compiled with -ffp-contract=off so
that no multiply-add is fused (the CUDA library is built with -fmad=false; both
sides then evaluate the same IEEE-754 operation sequences).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["rng_math.cpp", "resample.cpp", "pl.cpp", "api.cpp"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h", "build.py"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force=False):
    """Compile liboracle.so if missing or older than its sources; return its path."""
    if not force and not _stale():
        return LIB
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
