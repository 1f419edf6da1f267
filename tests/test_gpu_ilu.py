"""ILU(0) local solvers of the fluid Schwarz blocks on the device (Sec. 3.3,
4.1; LU stays for the solid blocks), mixed precision, against the oracle's
V-cycle with the same local solvers: one V-cycle within FP32 accuracy
(1e-3 relative, as for the exact-inverse mixed path), and the Newton
correction within 1e-8 of the oracle's direct solution with the FGMRES
iteration count within 10 % (at least 1) of the oracle's; 2D and 3D."""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import solver as osolver  # noqa: E402
from oracle.mesh import initial_state  # noqa: E402
from paper_1709_05660_gb300.workloads import CONFIGS, noise  # noqa: E402


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("tile", [(2, 2), (4, 4)], ids=["2x2", "4x4"])
def test_fluid_ilu_vcycle_and_newton_step(tile):
    from paper_1709_05660_gb300 import fsi
    torch.cuda.set_device(0)
    prob, opts = CONFIGS["channel2d_l3"]
    opts = replace(opts, precision=1, local_solver=1, tile=tile)
    orc = osolver.Oracle(prob, opts)
    N = orc.fine.N
    y0 = initial_state(prob, orc.fine, noise(N, 0))
    r, J = orc.assemble(y0)
    orc.factor()
    xs = osolver.direct_solve(J, -r)
    _, sto = orc.solve(-r)
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        s.set_state(_dev(y0))
        s.assemble()
        s.factor()
        b = np.random.default_rng(3).standard_normal(N)
        z = torch.empty(N, dtype=torch.float64, device="cuda")
        s.apply_vcycle(_dev(b), z)
        want = orc.precond(b)
        assert np.linalg.norm(z.cpu().numpy() - want) <= 1e-3 * np.linalg.norm(want)
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.set_state(_dev(y0))
        _, st = s.newton_step(dx)
        err = np.linalg.norm(dx.cpu().numpy() - xs) / np.linalg.norm(xs)
        assert err <= 1e-8, err
        assert abs(st.iters - sto.iters) <= max(1, int(0.1 * sto.iters)), (st.iters, sto.iters)
    finally:
        s.close()


def test_fluid_ilu_needs_mixed_precision():
    from paper_1709_05660_gb300 import fsi
    prob, opts = CONFIGS["channel2d_l3"]
    with pytest.raises(fsi.FSIError) as ei:
        fsi.FSI(replace(prob, levels=2), replace(opts, precision=0, local_solver=1),
                stream=torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == -1


def test_fluid_ilu_3d_newton_step():
    """The same bars on the small 3D box (2 x 2 x 2-element blocks, node
    blocks of 6 unknowns, element blocks of 4), mean inflow 0.2."""
    from paper_1709_05660_gb300 import fsi
    from paper_1709_05660_gb300.workloads import SolverOpts
    from tests.oracle_cases import SMALL_3D
    torch.cuda.set_device(0)
    prob = replace(SMALL_3D, levels=2, U=0.2)
    opts = SolverOpts(tile=(2, 2, 2), precision=1, local_solver=1)
    orc = osolver.Oracle(prob, opts)
    N = orc.fine.N
    y0 = initial_state(prob, orc.fine, noise(N, 0))
    r, J = orc.assemble(y0)
    orc.factor()
    xs = osolver.direct_solve(J, -r)
    _, sto = orc.solve(-r)
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        s.set_state(_dev(y0))
        s.assemble()
        s.factor()
        b = np.random.default_rng(4).standard_normal(N)
        z = torch.empty(N, dtype=torch.float64, device="cuda")
        s.apply_vcycle(_dev(b), z)
        want = orc.precond(b)
        assert np.linalg.norm(z.cpu().numpy() - want) <= 1e-3 * np.linalg.norm(want)
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.set_state(_dev(y0))
        _, st = s.newton_step(dx)
        err = np.linalg.norm(dx.cpu().numpy() - xs) / np.linalg.norm(xs)
        assert err <= 1e-8, err
        assert abs(st.iters - sto.iters) <= max(1, int(0.1 * sto.iters)), (st.iters, sto.iters)
    finally:
        s.close()
