"""The bounds-check build (libfsi_bounds.so, -DFSI_BOUNDS_CHECK), the test
suite's substitute for a memory sanitizer: index checks in the Schwarz
gather, apply, factorisation and ILU(0) kernels and in the block-sparse and
coarse gathers record the first failing site and skip the access; a call then
returns FSI_E_CUDA naming the site.  Here the checked library runs Newton
steps of the 2D channel (FP64 and mixed precision, exact inverses and ILU(0)
fluid blocks) and of the small 3D box in a child process: every call returns
FSI_OK (no check fired) and the corrections match the oracle's direct
solutions at the usual bars."""
import os
import subprocess
import sys
import tempfile
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from dataclasses import replace
from paper_1709_05660_gb300 import fsi
from paper_1709_05660_gb300.workloads import CONFIGS, SolverOpts, noise
from tests.oracle_cases import SMALL_3D
fsi.load_library(sys.argv[2])
torch.cuda.set_device(0)
prob2, opts2 = CONFIGS["channel2d_l3"]
cases = {"fp64": (prob2, opts2), "mixed": (prob2, replace(opts2, precision=1)),
         "ilu": (replace(prob2, U=0.2), replace(opts2, precision=1, local_solver=1)),
         "box3d": (replace(SMALL_3D, levels=2), SolverOpts(tile=(2, 2, 2), precision=1))}
out = {}
for name, (prob, opts) in cases.items():
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream, tuned=False)
    N = int(s.N[-1])
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    s.initial_state(torch.tensor(noise(N, 0), dtype=torch.float64, device="cuda"), y)
    s.set_state(y)
    dx = torch.empty(N, dtype=torch.float64, device="cuda")
    s.newton_step(dx)
    out[name] = dx.cpu().numpy()
    s.close()
np.savez(sys.argv[3], **out)
'''


def test_bounds_checked_library_runs_clean():
    from paper_1709_05660_gb300 import build as fbuild
    from paper_1709_05660_gb300.workloads import CONFIGS, SolverOpts, noise
    from oracle import solver as osolver
    from oracle.mesh import initial_state
    from tests.oracle_cases import SMALL_3D
    lib = fbuild.build(bounds_check=True)
    with tempfile.TemporaryDirectory() as td:
        res = os.path.join(td, "dx.npz")
        p = subprocess.run([sys.executable, "-c", CHILD, ROOT, lib, res], capture_output=True, text=True,
                           timeout=900)
        assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
        got = dict(np.load(res))
    prob2, opts2 = CONFIGS["channel2d_l3"]
    cases = {"fp64": (prob2, opts2, 1e-10), "mixed": (prob2, replace(opts2, precision=1), 1e-8),
             "ilu": (replace(prob2, U=0.2), replace(opts2, precision=1, local_solver=1), 1e-8),
             "box3d": (replace(SMALL_3D, levels=2), SolverOpts(tile=(2, 2, 2), precision=1), 1e-8)}
    for name, (prob, opts, tol) in cases.items():
        orc = osolver.Oracle(prob, opts)
        y0 = initial_state(prob, orc.fine, noise(orc.fine.N, 0))
        r, J = orc.assemble(y0)
        xs = osolver.direct_solve(J, -r)
        err = np.linalg.norm(got[name] - xs) / np.linalg.norm(xs)
        assert err <= tol, (name, err)
