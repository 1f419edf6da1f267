"""Builds libfsi.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel, then linked into
``paper_1709_05660_gb300/libfsi.so``.  Usage: ``python -m
paper_1709_05660_gb300.build [--bounds-check]`` or ``build()`` from Python;
``--bounds-check`` builds ``libfsi_bounds.so`` with index checks in the
kernels (the sanitizer substitute of the test suite).
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libfsi.so")
BOUNDS_OUT = os.path.join(HERE, "libfsi_bounds.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(verbose: bool = False, extra_flags=(), bounds_check: bool = False) -> str:
    """Builds libfsi.so, or with bounds_check the bounds-check variant
    libfsi_bounds.so (-DFSI_BOUNDS_CHECK: index checks in the gather, apply,
    factorisation and sparse-product kernels that record the failing site and
    skip the access; calls then return FSI_E_CUDA naming the site)."""
    nvcc = _nvcc()
    out = BOUNDS_OUT if bounds_check else OUT
    build_dir = BUILD_DIR + ("_bounds" if bounds_check else "")
    if bounds_check:
        extra_flags = tuple(extra_flags) + ("-DFSI_BOUNDS_CHECK",)
    os.makedirs(build_dir, exist_ok=True)
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    common = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I" + os.path.join(HERE, "..", "include")]
    jobs = []
    for f in cu:
        obj = os.path.join(build_dir, f + ".o")
        jobs.append([nvcc, ARCH, "-lineinfo", "--expt-relaxed-constexpr", *common, *extra_flags,
                     "-c", os.path.join(CSRC, f), "-o", obj])
    for f in cpp:
        obj = os.path.join(build_dir, f + ".o")
        jobs.append([nvcc, *common, *(["-DFSI_BOUNDS_CHECK"] if bounds_check else []), "-x", "c++", "-c",
                     os.path.join(CSRC, f), "-o", obj])
    with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(build_dir, f + ".o") for f in cu + cpp]
    tmp = out + ".tmp"
    _run([nvcc, ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    flags = [f for f in sys.argv[1:] if f != "--bounds-check"]
    print(build(verbose=True, extra_flags=flags, bounds_check="--bounds-check" in sys.argv[1:]))
