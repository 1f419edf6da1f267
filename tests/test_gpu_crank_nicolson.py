"""GPU parity of the paper's Crank-Nicolson time step (Sec. 2.5, with the
conservative ALE identity of Sec. 2.3) against the CPU oracle: the 3-level
2D channel and the 2-level 3D box, one step dt = 0.01 at t = 0.13 from a
perturbed t_n state (nonzero mesh velocity).  Same bars as the BDF tests:
residual and finest Jacobian within 1e-12 of each row's largest entry,
Galerkin levels within 1e-10, the Newton correction within 1e-10 of the
oracle's direct solution on the FP64 path (solved to rtol 1e-12) and 1e-8 on
the mixed path."""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import solver as osolver  # noqa: E402
from oracle.mesh import initial_state  # noqa: E402
from paper_1709_05660_gb300.workloads import CONFIGS, SolverOpts, noise  # noqa: E402
from tests.oracle_cases import SMALL_3D  # noqa: E402
from tests.test_gpu_transient import _csr, _dev, _rows_close  # noqa: E402


def _case(prob, opts, seed):
    orc = osolver.Oracle(prob, opts)
    N = orc.fine.N
    rng = np.random.default_rng(seed)
    free = ~orc.fine.dir_mask
    y = initial_state(prob, orc.fine, noise(N, 3))
    yn = y + 1e-4 * rng.standard_normal(N) * free
    t = 0.13
    r, J = orc.assemble(y, tr=dict(scheme="cn", yn=yn, dt=prob.dt, t=t))
    return orc, y, yn, t, r, J, osolver.direct_solve(J, -r)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_cn_step_parity_2d(precision):
    from paper_1709_05660_gb300 import fsi
    torch.cuda.set_device(0)
    prob, opts = CONFIGS["channel2d_l3"]
    prob = replace(prob, transient=2, dt=0.01, mr_c2=0.1 * prob.mu_s)
    opts = replace(opts, rtol=1e-12, precision=precision)
    orc, y, yn, t, r, J, xs = _case(prob, opts, 50)
    N = len(y)
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        s.set_state(_dev(y), _dev(yn), None, t)
        rg = torch.empty(N, dtype=torch.float64, device="cuda")
        s.assemble(rg)
        assert np.max(np.abs(rg.cpu().numpy() - r)) <= 1e-12 * np.max(np.abs(r))
        L = prob.levels
        _rows_close(_csr(s, L - 1), J, 1e-12)
        for l in range(L - 1):
            _rows_close(_csr(s, l), orc.ops[l].J, 1e-10)
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.set_state(_dev(y), _dev(yn), None, t)
        s.newton_step(dx)
        err = np.linalg.norm(dx.cpu().numpy() - xs) / np.linalg.norm(xs)
        assert err <= (1e-10 if precision == 0 else 1e-8), err
    finally:
        s.close()


def test_cn_step_parity_3d():
    from paper_1709_05660_gb300 import fsi
    prob = replace(SMALL_3D, levels=2, transient=2, dt=0.01)
    opts = SolverOpts(tile=(2, 2, 2), precision=0, rtol=1e-12)
    orc, y, yn, t, r, J, xs = _case(prob, opts, 51)
    N = len(y)
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        s.set_state(_dev(y), _dev(yn), None, t)
        rg = torch.empty(N, dtype=torch.float64, device="cuda")
        s.assemble(rg)
        assert np.max(np.abs(rg.cpu().numpy() - r)) <= 1e-12 * np.max(np.abs(r))
        _rows_close(_csr(s, prob.levels - 1), J, 1e-12)
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.set_state(_dev(y), _dev(yn), None, t)
        s.newton_step(dx)
        err = np.linalg.norm(dx.cpu().numpy() - xs) / np.linalg.norm(xs)
        assert err <= 1e-10, err
    finally:
        s.close()
