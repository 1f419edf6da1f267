"""GPU parity of the transient (BDF) form against the CPU oracle.

Channel-with-flap geometry of the 2D benchmark at three levels, one time step
dt = 0.01 at t = 0.13 (inflow amplitude alpha(t) < 1), BDF1 (start-up step)
and BDF2.  Same bars as the steady parity tests: residual and finest Jacobian
entries within 1e-12 of their row's largest magnitude, Galerkin levels within
1e-10, the Newton correction within 1e-10 relative of the oracle's direct
solution.  The mass terms change the conditioning: a true residual of 1e-10
left an error of 2.2e-10 against the direct solution, so the solve here runs
to rtol 1e-12, which bounds the error well inside 1e-10.
"""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import fem, solver as osolver  # noqa: E402
from oracle.mesh import initial_state  # noqa: E402
from paper_1709_05660_gb300.workloads import CONFIGS, noise  # noqa: E402


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rows_close(Ag, Ao, tol):
    D = (Ag - Ao).tocsr()
    rowmax = abs(Ao.tocsr()).max(axis=1).toarray().ravel()
    rowmax[rowmax == 0] = 1.0
    worst = float(np.max(abs(D).max(axis=1).toarray().ravel() / rowmax))
    assert worst <= tol, worst


def _csr(s, level):
    import scipy.sparse as sp
    rp, c, v = s.export_csr(level)
    n = len(rp) - 1
    return sp.csr_matrix((v, c, rp), shape=(n, n))


@pytest.mark.parametrize("order", [1, 2], ids=["bdf1", "bdf2"])
def test_transient_step_parity(order):
    from paper_1709_05660_gb300 import fsi
    torch.cuda.set_device(0)
    prob, opts = CONFIGS["channel2d_l3"]
    prob = replace(prob, transient=1, dt=0.01)
    opts = replace(opts, rtol=1e-12)
    orc = osolver.Oracle(prob, opts)
    N = orc.fine.N
    rng = np.random.default_rng(40 + order)
    y = initial_state(prob, orc.fine, noise(N, 3))
    yn = y + 1e-4 * rng.standard_normal(N)
    ynm1 = yn + 1e-4 * rng.standard_normal(N)
    t = 0.13
    tr = dict(yn=yn, ynm1=ynm1 if order == 2 else np.zeros(N), a=fem.bdf_coefficients(order), dt=prob.dt, t=t)
    r, J = orc.assemble(y, tr=tr)
    xs = osolver.direct_solve(J, -r)

    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        s.set_state(_dev(y), _dev(yn), _dev(ynm1) if order == 2 else None, t)
        rg = torch.empty(N, dtype=torch.float64, device="cuda")
        s.assemble(rg)
        rg = rg.cpu().numpy()
        assert np.max(np.abs(rg - r)) <= 1e-12 * np.max(np.abs(r))
        L = prob.levels
        _rows_close(_csr(s, L - 1), J, 1e-12)
        for l in range(L - 1):
            _rows_close(_csr(s, l), orc.ops[l].J, 1e-10)
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.set_state(_dev(y), _dev(yn), _dev(ynm1) if order == 2 else None, t)
        _, st = s.newton_step(dx)
        err = np.linalg.norm(dx.cpu().numpy() - xs) / np.linalg.norm(xs)
        assert err <= 1e-10, (err, st.iters)
    finally:
        s.close()


def test_transient_needs_history():
    from paper_1709_05660_gb300 import fsi
    prob, opts = CONFIGS["channel2d_l3"]
    prob = replace(prob, transient=1, dt=0.01, levels=2)
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        N = int(s.N[-1])
        y = torch.zeros(N, dtype=torch.float64, device="cuda")
        with pytest.raises(fsi.FSIError):
            s.set_state(y)                 # y_prev missing
        with pytest.raises(fsi.FSIError):
            s.assemble()                   # no history yet
    finally:
        s.close()
