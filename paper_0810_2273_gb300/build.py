"""Build libvdwdf.so in-tree (paper_0810_2273_gb300/_build/) for sm_103a.

Each CUDA translation unit is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo``; the host table builder
by g++ with OpenMP; nvcc links the shared library (static CUDA runtime).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libvdwdf.so")

CU_SOURCES = ["api.cu", "pair.cu", "prep.cu", "assemble.cu", "spectral.cu", "tail.cu", "peak.cu"]
CXX_SOURCES = ["table.cpp"]
HEADERS = ["common.cuh", "table.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in CU_SOURCES + CXX_SOURCES + HEADERS]
    deps += [os.path.join(INCLUDE, "vdwdf.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile and link libvdwdf.so if missing or out of date; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for s in CU_SOURCES:
        obj = os.path.join(OUT_DIR, s + ".o")
        cmd = [nvcc] + ARCH + common + ["-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills",
                                        "-c", os.path.join(CSRC, s), "-o", obj]
        jobs.append((cmd, obj))
    for s in CXX_SOURCES:
        obj = os.path.join(OUT_DIR, s + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", "-I", INCLUDE, "-I", CSRC,
               "-c", os.path.join(CSRC, s), "-o", obj]
        jobs.append((cmd, obj))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed:\n%s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
        return p.stdout + p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(run, [c for c, _ in jobs]))
    if verbose:
        for l in logs:
            if l.strip():
                print(l, file=sys.stderr)
    tmp = LIB + ".tmp%d" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for _, o in jobs] + ["-Xcompiler", "-fopenmp", "-lgomp"]
    run(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
