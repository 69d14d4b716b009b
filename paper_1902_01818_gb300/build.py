"""Builds libmgiga.so in-tree for sm_103a (GB300).

Host set-up sources (C++17, OpenMP) are compiled with g++, device sources with
nvcc, all translation units in parallel; the shared library is linked by nvcc
with the static CUDA runtime.  Objects go to _build/, the library to _lib/.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libmgiga.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SOURCES = ["host_spline.cpp", "host_assembly.cpp", "host_hierarchy.cpp", "host_problem.cpp", "tune.cpp"]
DEVICE_SOURCES = ["kernels.cu", "gs_staged_2d.cu", "gs_staged_3d.cu", "fd_fused.cu", "fd_cluster.cu", "setup_gpu.cu", "matfree.cu", "solver.cu"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmgiga")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".hpp", ".cuh"))]
    return hs + [os.path.join(INCLUDE, "mgiga.h")]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(x) > t for x in [src] + _headers())


def _compile(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("compilation failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    return res.stdout + res.stderr


def build(verbose=False, force=False):
    """Compile and link libmgiga.so if any source changed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src in HOST_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, s):
            jobs.append(["g++", "-std=c++17", "-O3", "-fopenmp", "-fPIC", "-Wall", "-Wno-unused-variable",
                         "-I", INCLUDE, "-c", s, "-o", o])
    for src in DEVICE_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, s):
            jobs.append([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
                                         "-I", INCLUDE, "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for out in ex.map(_compile, jobs):
            if verbose and out.strip():
                print(out)
    relink = force or bool(jobs) or not os.path.exists(LIB)
    if relink:
        tmp = LIB + ".tmp"
        # --no-undefined: a launcher missing from the objects fails the build, not the import
        _compile([nvcc] + ARCH + ["-shared", "-o", tmp] + objs +
                 ["-Xcompiler", "-fopenmp", "-lgomp", "-Xlinker", "--no-undefined", "-lpthread", "-ldl", "-lrt"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
