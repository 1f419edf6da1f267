"""Error paths of the C-ABI, each produced by an allowed form (nothing faults,
traps or hangs the GPU): an iteration cap, a defective operator imported on
the host, and a tensor-core wait whose limit is set so short that it gives
up before the work it waits for has finished.  After each error the instance
stays usable and reproduces the oracle's Newton correction.
"""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import solver as osolver  # noqa: E402
from oracle.mesh import initial_state  # noqa: E402
from paper_1709_05660_gb300.workloads import CONFIGS, noise  # noqa: E402

E_SINGULAR, E_NOT_CONVERGED, E_TIMEOUT = -4, -5, -8


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ref():
    prob, opts = CONFIGS["channel2d_l3"]
    orc = osolver.Oracle(prob, opts)
    y0 = initial_state(prob, orc.fine, noise(orc.fine.N, 0))
    r, J = orc.assemble(y0)
    return dict(prob=prob, opts=opts, y0=y0, r=r, xs=osolver.direct_solve(J, -r), N=orc.fine.N)


def _instance(ref, **kw):
    from paper_1709_05660_gb300 import fsi
    torch.cuda.set_device(0)
    s = fsi.FSI(ref["prob"], replace(ref["opts"], **kw), stream=torch.cuda.current_stream().cuda_stream)
    s.set_state(_dev(ref["y0"]))
    return s


def _step_error(s, ref):
    dx = torch.empty(ref["N"], dtype=torch.float64, device="cuda")
    s.set_state(_dev(ref["y0"]))
    s.newton_step(dx)
    d = dx.cpu().numpy()
    return np.linalg.norm(d - ref["xs"]) / np.linalg.norm(ref["xs"])


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_not_converged_fills_stats(ref, precision):
    """FGMRES capped at 2 iterations: FSI_E_NOT_CONVERGED with the statistics
    filled (2 iterations, the true residual of the partial solution)."""
    from paper_1709_05660_gb300 import fsi
    s = _instance(ref, precision=precision, max_iters=2)
    try:
        r = torch.empty(ref["N"], dtype=torch.float64, device="cuda")
        s.assemble(r)
        s.factor()
        x = torch.zeros(ref["N"], dtype=torch.float64, device="cuda")
        with pytest.raises(fsi.FSIError) as ei:
            s.solve(-r, x)
        assert ei.value.code == E_NOT_CONVERGED
        st = ei.value.stats
        assert st.iters == 2
        assert ref["opts"].rtol < st.rel_res < 1.0
        # the partial solution is returned and its true residual is the reported one
        J = None
        rg = r.cpu().numpy()
        import scipy.sparse as sp
        rp, c, v = s.export_csr(ref["prob"].levels - 1)
        J = sp.csr_matrix((v, c, rp), shape=(ref["N"], ref["N"]))
        xr = x.cpu().numpy()
        assert np.linalg.norm(rg + J @ xr) / np.linalg.norm(rg) == pytest.approx(st.rel_res, rel=1e-6)
        with pytest.raises(fsi.FSIError) as ei:
            s.newton_step()
        assert ei.value.code == E_NOT_CONVERGED
    finally:
        s.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_singular_schwarz_block(ref, precision):
    """A zero column imported into the finest operator makes the Schwarz
    blocks that contain that unknown singular: FSI_E_SINGULAR from the
    factorisation.  Re-assembling restores the operator and the next Newton
    step matches the oracle."""
    from paper_1709_05660_gb300 import fsi
    s = _instance(ref, precision=precision)
    try:
        L = ref["prob"].levels
        s.assemble()
        rp, c, v = s.export_csr(L - 1)
        col = 4 * 200 + 3                   # u_y of an interior fluid node
        v = v.copy()
        v[c == col] = 0.0
        s.import_csr(L - 1, v)
        with pytest.raises(fsi.FSIError) as ei:
            s.factor()
        assert ei.value.code == E_SINGULAR
        assert _step_error(s, ref) <= (1e-10 if precision == 0 else 1e-8)
    finally:
        s.close()


def test_tensor_core_wait_timeout(ref):
    """The first wait of every block of the tensor-core factorisation given a
    limit of zero iterations gives up at once: each block then waits (with the
    full limit) for the UMMAs it has issued, releases its tensor memory and
    the call returns FSI_E_TIMEOUT.  With the built-in limit restored the same
    instance factors and solves as before."""
    from paper_1709_05660_gb300 import fsi
    s = _instance(ref, precision=1)
    try:
        s.assemble()
        s.set_tc_wait_limit(0)
        with pytest.raises(fsi.FSIError) as ei:
            s.factor()
        assert ei.value.code == E_TIMEOUT
        s.set_tc_wait_limit(-1)
        s.factor()
        assert _step_error(s, ref) <= 1e-8
    finally:
        s.close()


def test_import_roundtrip_reproduces_the_step(ref):
    """Exporting and importing the assembled operator changes nothing: the
    factorisation and solve on the imported values give the same correction
    bit for bit."""
    s = _instance(ref, precision=0)
    try:
        L = ref["prob"].levels
        r = torch.empty(ref["N"], dtype=torch.float64, device="cuda")
        s.assemble(r)
        s.factor()
        x0 = torch.zeros(ref["N"], dtype=torch.float64, device="cuda")
        s.solve(-r, x0)
        for l in range(L):
            s.import_csr(l, s.export_csr(l)[2])
        s.factor()
        x1 = torch.zeros(ref["N"], dtype=torch.float64, device="cuda")
        s.solve(-r, x1)
        assert torch.equal(x0, x1)
    finally:
        s.close()
