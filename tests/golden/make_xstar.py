"""Writes the oracle's Newton-step solutions at the benchmark sizes.

For each 2D channel workload at its seeded linearisation state y0 (the
benchmark state: inflow-profile velocity, N(0, 1e-4^2) noise on the free
displacements, seed 0) this computes, with the CPU oracle only:

* r(y0), the exact Jacobian J(y0) and the Galerkin hierarchy (Sec. 2.3, 3.2);
* x* = J^{-1}(-r): the oracle's sparse direct solve (LU + iterative
  refinement) where it fits in memory and time, else the oracle's own
  FGMRES with the V-cycle driven to a true relative residual of 1e-13
  (the plain definition of the Newton-step solve, Sec. 3.1);
* the oracle FGMRES(30) iteration counts at the workload's tolerance and at
  a ten times tighter one (Sec. 4.1 with this build's FGMRES reading), for
  iteration-count parity of the mixed and the FP64 path;
* a seeded sample of rows of every Galerkin level J_l, l < L-1, as
  (row, column, value) triples, for sampled parity of the coarse operators.

Output: ``tests/golden/xstar_<workload>.npz`` (compressed).  Nothing here
calls the CUDA path.

Usage: python tests/golden/make_xstar.py channel2d_l5 [channel2d_l6 ...]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solver as osolver  # noqa: E402
from oracle.mesh import initial_state  # noqa: E402
from paper_1709_05660_gb300.workloads import CONFIGS, noise  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
DIRECT_MAX_N = int(os.environ.get("XSTAR_DIRECT_MAX_N", "400000"))   # SuperLU fill / time stay modest below this
ROWS_PER_LEVEL = 48


def make(name: str) -> str:
    prob, opts = CONFIGS[name]
    t0 = time.time()
    orc = osolver.Oracle(prob, opts)
    lev = orc.fine
    y0 = initial_state(prob, lev, noise(lev.N, 0))
    r, J = orc.assemble(y0)
    t_asm = time.time() - t0
    print(f"{name}: N={lev.N} assembled in {t_asm:.0f} s", flush=True)
    t0 = time.time()
    orc.factor()
    x_it, st = orc.solve(-r, rtol=opts.rtol)
    iters, rel_it = st.iters, st.rel_res
    print(f"{name}: oracle FGMRES {iters} iterations to {rel_it:.2e} in {time.time() - t0:.0f} s", flush=True)
    _, st_t = orc.solve(-r, rtol=opts.rtol / 10)
    print(f"{name}: oracle FGMRES {st_t.iters} iterations to {st_t.rel_res:.2e} (rtol {opts.rtol / 10:g})", flush=True)
    t0 = time.time()
    if lev.N <= DIRECT_MAX_N:
        xs = osolver.direct_solve(J, -r)
        how = "sparse LU (SuperLU) + 2 steps of iterative refinement"
    else:
        xs, st2 = osolver.fgmres(J, -r, orc.precond, opts.restart, 1e-13, 2000)
        how = f"oracle FGMRES(30) + V-cycle to true rel. residual {st2.rel_res:.2e} ({st2.iters} iterations)"
    res = np.linalg.norm(r + J @ xs) / np.linalg.norm(r)
    print(f"{name}: x* by {how}, rel. residual {res:.2e}, {time.time() - t0:.0f} s", flush=True)
    # sampled rows of the Galerkin levels
    rng = np.random.default_rng(11)
    s_lv, s_row, s_col, s_val = [], [], [], []
    for l in range(prob.levels - 1):
        Jl = orc.ops[l].J.tocsr()
        rows = np.sort(rng.choice(Jl.shape[0], min(ROWS_PER_LEVEL, Jl.shape[0]), replace=False))
        for i in rows:
            a, b = Jl.indptr[i], Jl.indptr[i + 1]
            s_lv.append(np.full(b - a, l, dtype=np.int32))
            s_row.append(np.full(b - a, i, dtype=np.int64))
            s_col.append(Jl.indices[a:b].astype(np.int64))
            s_val.append(Jl.data[a:b].copy())
    out = os.path.join(HERE, f"xstar_{name}.npz")
    np.savez_compressed(
        out, xstar=xs, oracle_iters=np.int64(iters), oracle_rel_res=np.float64(rel_it),
        oracle_rtol=np.float64(opts.rtol), oracle_iters_tight=np.int64(st_t.iters),
        oracle_rtol_tight=np.float64(opts.rtol / 10),
        xstar_rel_res=np.float64(res), rnorm=np.float64(np.linalg.norm(r)), N=np.int64(lev.N),
        y0_checksum=np.float64(np.sum(y0 * np.arange(1, lev.N + 1) / lev.N)),
        how=np.array(how), galerkin_level=np.concatenate(s_lv), galerkin_row=np.concatenate(s_row),
        galerkin_col=np.concatenate(s_col), galerkin_val=np.concatenate(s_val))
    return out


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["channel2d_l5", "channel2d_l6"]:
        print(make(nm), flush=True)
