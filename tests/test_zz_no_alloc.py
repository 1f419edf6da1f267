"""fsi_coarse_solve_static: the coarse solve with its GEMV partial sums in a
file-scope device array.  Compared, two calls in a row, with the coarse step
of fsi_apply_vcycle on a one-level instance (same kernels and summation
order: equal bit for bit), checked against a sparse direct solve of the
oracle's level-0 operator, and its size limit.  This file is collected last
so that it also runs after every other GPU test has used the device.
"""
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


def _instance(prob, opts):
    from paper_1709_05660_gb300 import fsi
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    orc = osolver.Oracle(prob, opts)
    y0 = initial_state(prob, orc.fine, noise(orc.fine.N, 0))
    orc.assemble(y0)
    s.set_state(_dev(y0))
    s.assemble()
    s.factor()
    return s, orc


def test_static_coarse_solve_matches_vcycle_bitwise():
    import scipy.sparse.linalg as spla
    prob, opts = CONFIGS["channel2d_l3"]
    s, orc = _instance(replace(prob, levels=1), opts)
    try:
        n = int(s.N[0])
        b = np.random.default_rng(3).standard_normal(n)
        ref = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
        got = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
        for k in range(2):
            s.apply_vcycle(_dev(b), ref[k])
        for k in range(2):
            s.coarse_solve_static(_dev(b), got[k])
        for k in range(2):
            assert torch.equal(got[k], ref[0]) and torch.equal(ref[k], ref[0])
        want = spla.spsolve(orc.ops[0].J.tocsc(), b)
        err = np.linalg.norm(got[0].cpu().numpy() - want) / np.linalg.norm(want)
        assert err <= 1e-10, err
        # host buffers are staged by the call itself
        xh = np.empty(n)
        s.coarse_solve_static(b.copy(), xh)
        assert np.array_equal(xh, got[0].cpu().numpy())
    finally:
        s.close()


def test_static_coarse_solve_on_a_hierarchy():
    """Level 0 of a three-level instance holds the Galerkin operator."""
    import scipy.sparse.linalg as spla
    prob, opts = CONFIGS["channel2d_l3"]
    s, orc = _instance(prob, opts)
    try:
        n = int(s.N[0])
        b = np.random.default_rng(4).standard_normal(n)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        s.coarse_solve_static(_dev(b), x)
        want = spla.spsolve(orc.ops[0].J.tocsc(), b)
        err = np.linalg.norm(x.cpu().numpy() - want) / np.linalg.norm(want)
        assert err <= 1e-9, err
    finally:
        s.close()


def test_static_coarse_solve_size_limit():
    """A coarse level above FSI_STATIC_COARSE_MAX (4096) is rejected before
    any launch; the instance stays usable."""
    from paper_1709_05660_gb300 import fsi
    prob, opts = CONFIGS["channel2d_l3"]
    xb = tuple(np.linspace(0.0, 2.0, 33))          # 32 x 8 coarse cells: 5,444 internal unknowns
    yb = tuple(np.linspace(0.0, 0.5, 9))
    big = replace(prob, levels=1, breaks=(xb, yb))
    s = fsi.FSI(big, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        n = int(s.N[0])
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        with pytest.raises(fsi.FSIError) as ei:
            s.coarse_solve_static(b, x)
        assert ei.value.code == -1 and "4096" in str(ei.value)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        s.initial_state(_dev(noise(n, 0)), y)
    finally:
        s.close()


def test_static_coarse_solve_needs_factors():
    """Before the first fsi_factor_schwarz the dense coarse inverse does not
    exist yet: the call is rejected (FSI_E_INVALID) instead of applying an
    uninitialised inverse."""
    from paper_1709_05660_gb300 import fsi
    prob, opts = CONFIGS["channel2d_l3"]
    s = fsi.FSI(replace(prob, levels=1), opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        n = int(s.N[0])
        b = torch.ones(n, dtype=torch.float64, device="cuda")
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        with pytest.raises(fsi.FSIError) as ei:
            s.coarse_solve_static(b, x)
        assert ei.value.code == -1 and "factor" in str(ei.value)
    finally:
        s.close()
