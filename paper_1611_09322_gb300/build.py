"""In-tree build of the native libraries (no cmake, no torch extension machinery).

    _build/libpse.so            CUDA sampler, C ABI of include/pse.h (nvcc, sm_103a)
    _build/libpse_workloads.so  seeded configuration generators (gcc)

Translation units are compiled in parallel, then linked.  Rebuilds only
when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build_workloads():
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(CSRC, "workloads.c")
    lib = os.path.join(OUT, "libpse_workloads.so")
    if _stale(lib, [src]):
        tmp = lib + ".tmp%d" % os.getpid()
        _run(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, lib)
    return lib


def cuda_sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def build_cuda(verbose=False):
    """Compile csrc/*.cu for sm_103a and link _build/libpse.so against cuFFT."""
    os.makedirs(OUT, exist_ok=True)
    lib = os.path.join(OUT, "libpse.so")
    srcs = cuda_sources()
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    if not _stale(lib, srcs + hdrs + [__file__]):
        return lib
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
                    "-I" + CSRC, "--expt-relaxed-constexpr", "-rdc=false"]
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        if _stale(obj, [src] + hdrs + [__file__]):
            out = _run([NVCC] + flags + ["-c", src, "-o", obj])
            if verbose and out:
                sys.stdout.write(out)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp%d" % os.getpid()
    _run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcufft", "-lcudart"])
    os.replace(tmp, lib)
    return lib


def build_all(verbose=False):
    return build_cuda(verbose), build_workloads()


if __name__ == "__main__":
    print(build_all(verbose="-v" in sys.argv))
