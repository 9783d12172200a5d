"""Build libdd.so (the CUDA library behind include/dd.h) for sm_103a, in-tree.

The translation units are compiled in parallel with nvcc and linked into
paper_2209_13168_gb300/libdd.so.  -fmad=false keeps every binary32 add and
multiply a separate rounding (the kernels also use __fmul_rn/__fadd_rn
explicitly); -prec-div/-prec-sqrt keep IEEE division and square root.
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libdd.so")
LIB_CHECKED = os.path.join(PKG, "libdd_checked.so")   # -DDD_CHECKED: index tests in the kernels
SOURCES = ["dd_kernels.cu", "dd_api.cu", "dd_serve.cu", "dd_noalloc.cu", "dd_mlp.cu", "dd_probe.cu", "dd_fast.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
           "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INCLUDE]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdd.so")


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, checked=False):
    """Compile libdd.so (checked=True: libdd_checked.so, with the kernels'
    index tests) if any source is newer; returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    cc = nvcc()
    bdir = os.path.join(PKG, "_build_checked" if checked else "_build")
    os.makedirs(bdir, exist_ok=True)
    flags = NVFLAGS + (["-DDD_CHECKED"] if checked else [])

    def compile_one(src):
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + ARCH + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        for _, log in results:
            print(log)
    return lib


if __name__ == "__main__":
    build(force=True, verbose=True)
