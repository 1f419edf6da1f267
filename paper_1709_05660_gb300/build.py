"""Builds libfsi.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel, then linked into
``paper_1709_05660_gb300/libfsi.so``.  Usage: ``python -m
paper_1709_05660_gb300.build`` or ``build()`` from Python.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libfsi.so")
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


def build(verbose: bool = False, extra_flags=()) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    common = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I" + os.path.join(HERE, "..", "include")]
    jobs = []
    for f in cu:
        obj = os.path.join(BUILD_DIR, f + ".o")
        jobs.append([nvcc, ARCH, "-lineinfo", "--expt-relaxed-constexpr", *common, *extra_flags,
                     "-c", os.path.join(CSRC, f), "-o", obj])
    for f in cpp:
        obj = os.path.join(BUILD_DIR, f + ".o")
        jobs.append([nvcc, *common, "-x", "c++", "-c", os.path.join(CSRC, f), "-o", obj])
    with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD_DIR, f + ".o") for f in cu + cpp]
    tmp = OUT + ".tmp"
    _run([nvcc, ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    flags = sys.argv[1:]
    print(build(verbose=True, extra_flags=flags))
