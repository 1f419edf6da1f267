"""The bounds-check variant of the kernels compiles for sm_103a (no GPU
needed: nvcc cross-compiles here); its checks are exercised on the GPU by
tests/test_gpu_bounds_build.py."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1709_05660_gb300", "csrc")


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_checked_kernels_compile():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as td:
        procs = [subprocess.Popen([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-std=c++17", "-O3",
                                   "--expt-relaxed-constexpr", "-DFSI_BOUNDS_CHECK",
                                   "-I" + os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, f),
                                   "-o", os.path.join(td, f + ".o")],
                                  stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
                 for f in ("k_linalg.cu", "k_schwarz.cu")]
        for p in procs:
            out, _ = p.communicate(timeout=600)
            assert p.returncode == 0, out[-3000:]
