"""Build libpf.so (the CUDA library behind include/pf.h) in-tree with nvcc.

Flags: sm_103a only; -fmad=false keeps every floating-point multiply and add
separately rounded, which (with IEEE division / square root and no
flush-to-zero, the defaults) makes the per-particle arithmetic a
deterministic sequence of IEEE-754 operations.
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libpf.so")
SOURCES = ["api.cu", "batch_f32.cu", "batch_f64.cu"]
DEPS = ["api.cu", "batch_f32.cu", "batch_f64.cu", "kernels.cuh", "device.cuh", "batch.cuh",
        "batch_launch.h", "batch_kernels.cuh", "batch_api.cuh", "server_api.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    files = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(INCLUDE, "pf.h"), __file__]
    return any(os.path.getmtime(f) > t for f in files)


def build(force=False, verbose=False):
    """Compile libpf.so if missing or stale; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(os.path.join(HERE, "_build"), exist_ok=True)
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(HERE, "_build", src.replace(".cu", ".o"))
        cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
               "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    for p, cmd in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.run([nvcc(), ARCH, "-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
