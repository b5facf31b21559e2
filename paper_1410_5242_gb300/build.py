"""Builds libkpm.so in-tree (paper_1410_5242_gb300/_build/) for sm_103a.

Each translation unit compiles in its own process (nvcc for .cu, g++ for
.cpp) and the objects are linked with nvcc into one shared library with the
CUDA runtime linked statically, so it loads next to any PyTorch build.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libkpm.so")
# the checked build (-DKPM_CHECK: bounds checks in the staged sweep)
BUILD_CHECK = os.path.join(PKG, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libkpm_check.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

SOURCES = ["kpm_host.cpp", "kpm_part.cpp", "kpm_ctx.cu", "kpm_batch.cu", "kpm_naive.cu", "aug_spmmv_fp64.cu",
           "aug_spmmv_fp32.cu", "aug_spmmv_staged.cu"]
HEADERS = ["kpm_internal.h", "aug_spmmv.cuh", os.path.join(INCLUDE, "kpm.h")]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkpm")


def _newest_input():
    paths = [os.path.join(CSRC, s) for s in SOURCES]
    paths += [h if os.path.isabs(h) else os.path.join(CSRC, h) for h in HEADERS]
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def _compile(src, extra, build_dir=BUILD):
    nvcc = _nvcc()
    obj = os.path.join(build_dir, src + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [nvcc, ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
               "-I" + INCLUDE, "-I" + CSRC, "-c", path, "-o", obj] + extra
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-I" + INCLUDE, "-I" + CSRC,
               "-I" + os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include"),
               "-c", path, "-o", obj] + [e for e in extra if e.startswith("-D")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compiling %s failed:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra_nvcc=(), check=False):
    """Compile and link libkpm.so (check: the checked build libkpm_check.so)
    if any source is newer; returns its path."""
    build_dir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    extra = list(extra_nvcc) + (["-DKPM_CHECK"] if check else [])
    os.makedirs(build_dir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, build_dir), SOURCES))
    if verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = lib + ".%d.tmp" % os.getpid()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "lib64")
    cmd = [_nvcc(), ARCH, "-shared", "-cudart", "static", "-o", tmp] + [o for o, _ in results] + \
        ["-L" + cuda_lib, "-lcusparse", "-lcublas", "-lpthread", "-Xlinker", "-rpath=" + cuda_lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("linking %s failed:\n%s" % (os.path.basename(lib), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, check="--check" in sys.argv))
