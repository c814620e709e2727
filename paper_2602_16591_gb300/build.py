"""Builds libpswf_ewald.so in-tree with nvcc for sm_103a (GB300).

Usage: ``python paper_2602_16591_gb300/build.py`` (runs without importing the package,
which needs the built library) or ``build()`` after loading this file.
Translation units are compiled in parallel; the shared library lands next to
this file so the Python binding loads it from the package directory.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libpswf_ewald.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "dispatch_f32.cu", "dispatch_f64.cu", "dispatch_ff.cu", "planner.cpp", "static_spread.cu", "batch_f32.cu",
           "tc_spread.cu"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src, verbose_ptxas=False):
    os.makedirs(BUILD, exist_ok=True)
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    # host code: no contraction of a*b+c into fma, so that x86-64 and AArch64 hosts round alike
    cmd = [_nvcc(), "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
           "-I" + os.path.join(ROOT, "include"),
           "-I" + CSRC, "-c", os.path.join(CSRC, src), "-o", obj] + ARCH
    if src.endswith(".cu"):
        cmd += ["--expt-relaxed-constexpr", "-Xcudafe", "--diag_suppress=177"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd += ["-x", "c++"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr[-8000:]))
    return obj, r.stderr


def build(verbose_ptxas=False, force=False):
    """Compile every translation unit and link libpswf_ewald.so (skips when up to date)."""
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "pswf_ewald.h")]
    if not force and os.path.exists(LIB):
        lib_t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= lib_t for d in deps) and not verbose_ptxas:
            return LIB
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    objs = [o for o, _ in results]
    cmd = [_nvcc(), "-shared", "-o", LIB] + objs + ARCH + ["-lcufft", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr[-8000:]))
    if verbose_ptxas:
        for (o, log), s in zip(results, SOURCES):
            sys.stderr.write("==== %s\n%s" % (s, log))
    return LIB


if __name__ == "__main__":
    build(verbose_ptxas="-v" in sys.argv, force=True)
    print(LIB)
