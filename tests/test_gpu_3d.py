"""GPU parity of the 3D device path (27-node hexahedra, 166 unknowns per
element, 6x6 node blocks, slab-blocked coarse LU) against the CPU oracle.

Workload: a 3 x 2 x 3 coarse box with the flap layer, two levels (6 x 4 x 6
fine hexahedra), Schwarz tiles 2 x 2 x 2.  Same bars as the 2D parity tests:
integer data bit-exact, finest residual / Jacobian within 1e-12 of each row's
largest magnitude, Galerkin level within 1e-10, smoother / V-cycle within the
backward-error bound of the equilibrated blocks, solutions within 1e-10 of
the oracle's direct solution (mixed path: 1e-8).
"""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import fem, solver as osolver  # noqa: E402
from oracle.mesh import initial_state  # noqa: E402
from paper_1709_05660_gb300.workloads import SolverOpts, noise  # noqa: E402
from tests.oracle_cases import SMALL_3D  # noqa: E402
from tests.test_gpu_parity import _block_cond, _csr, _rows_close  # noqa: E402

EPS = np.finfo(np.float64).eps
PROB = replace(SMALL_3D, levels=2)
OPTS = SolverOpts(tile=(2, 2, 2))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def c3d():
    from paper_1709_05660_gb300 import fsi
    torch.cuda.set_device(0)
    s = fsi.FSI(PROB, OPTS, stream=torch.cuda.current_stream().cuda_stream)
    orc = osolver.Oracle(PROB, OPTS)
    N = orc.fine.N
    y0 = initial_state(PROB, orc.fine, noise(N, 0))
    r, J = orc.assemble(y0)
    orc.factor()
    xs = osolver.direct_solve(J, -r)
    yield dict(s=s, orc=orc, y0=y0, r=r, J=J, xs=xs, N=N)
    s.close()


def test_3d_numbering_and_initial_state(c3d):
    s, orc = c3d["s"], c3d["orc"]
    assert int(s.N[-1]) == orc.fine.N and int(s.N[0]) == orc.levels_mesh[0].N
    y = torch.empty(c3d["N"], dtype=torch.float64, device="cuda")
    s.initial_state(_dev(noise(c3d["N"], 0)), y)
    assert np.array_equal(_host(y), c3d["y0"])


def test_3d_residual_jacobian_galerkin(c3d):
    s, orc = c3d["s"], c3d["orc"]
    s.set_state(_dev(c3d["y0"]))
    r = torch.empty(c3d["N"], dtype=torch.float64, device="cuda")
    s.assemble(r)
    assert np.max(np.abs(_host(r) - c3d["r"])) <= 1e-12 * np.max(np.abs(c3d["r"]))
    Jg = _csr(s, 1)
    assert np.array_equal(Jg.indptr, c3d["J"].indptr) and np.array_equal(Jg.indices, c3d["J"].indices)
    _rows_close(Jg, c3d["J"], 1e-12)
    _rows_close(_csr(s, 0), orc.ops[0].J, 1e-10)


def test_3d_smoother_and_vcycle(c3d):
    s, orc = c3d["s"], c3d["orc"]
    s.set_state(_dev(c3d["y0"]))
    s.assemble()
    s.factor()
    rng = np.random.default_rng(5)
    ops = orc.ops[1]
    cond, nmax = _block_cond(ops)
    n = ops.J.shape[0]
    b, x = rng.standard_normal(n), rng.standard_normal(n)
    want = x + OPTS.omega * osolver.ras_apply(ops, b - ops.J @ x)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    s.apply_smoother(1, _dev(b), _dev(x), out)
    err = np.linalg.norm(_host(out) - want) / np.linalg.norm(want)
    assert err <= 10 * nmax * EPS * cond, (err, cond)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    s.apply_vcycle(_dev(b), z)
    want = orc.precond(b)
    err = np.linalg.norm(_host(z) - want) / np.linalg.norm(want)
    assert err <= 100 * nmax * EPS * cond, (err, cond)


def test_3d_fgmres_and_newton_step(c3d):
    from paper_1709_05660_gb300 import fsi
    s, orc = c3d["s"], c3d["orc"]
    s.set_state(_dev(c3d["y0"]))
    s.assemble()
    s.factor()
    b = -c3d["r"]
    x = torch.zeros(c3d["N"], dtype=torch.float64, device="cuda")
    st = s.solve(_dev(b), x)
    err = np.linalg.norm(_host(x) - c3d["xs"]) / np.linalg.norm(c3d["xs"])
    assert err <= 1e-10, err
    _, sto = orc.solve(b)
    assert abs(st.iters - sto.iters) <= max(1, int(0.1 * sto.iters)), (st.iters, sto.iters)
    sm = fsi.FSI(PROB, replace(OPTS, precision=1), stream=torch.cuda.current_stream().cuda_stream)
    try:
        sm.set_state(_dev(c3d["y0"]))
        dx = torch.empty(c3d["N"], dtype=torch.float64, device="cuda")
        sm.newton_step(dx)
        err = np.linalg.norm(_host(dx) - c3d["xs"]) / np.linalg.norm(c3d["xs"])
        assert err <= 1e-8, err
    finally:
        sm.close()


@pytest.mark.parametrize("levels", [1, 2], ids=["coarse-only", "two-level"])
def test_3d_coarse_slab_solve(levels):
    """One level: the V-cycle is the slab-blocked coarse LU solve itself."""
    from paper_1709_05660_gb300 import fsi
    import scipy.sparse.linalg as spla
    prob = replace(SMALL_3D, levels=levels)
    s = fsi.FSI(prob, OPTS, stream=torch.cuda.current_stream().cuda_stream)
    try:
        orc = osolver.Oracle(prob, OPTS)
        y0 = initial_state(prob, orc.fine, noise(orc.fine.N, 1))
        orc.assemble(y0)
        s.set_state(_dev(y0))
        s.assemble()
        s.factor()
        J0 = orc.ops[0].J.tocsc()
        rng = np.random.default_rng(9)
        b = rng.standard_normal(J0.shape[0])
        want = spla.spsolve(J0, b)
        if levels == 1:
            z = torch.empty(len(b), dtype=torch.float64, device="cuda")
            s.apply_vcycle(_dev(b), z)
            got = _host(z)
        else:
            # level-0 operator of the device hierarchy applied to the exact
            # solution returns b (checks the Galerkin operator the LU factors)
            y = torch.empty(len(b), dtype=torch.float64, device="cuda")
            s.apply_operator(0, _dev(want), y)
            got = spla.spsolve(J0, _host(y))
        cond = np.linalg.cond(J0.toarray())
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= 1e3 * EPS * cond, (err, cond)
    finally:
        s.close()


def test_3d_transient_bdf2_step():
    from paper_1709_05660_gb300 import fsi
    prob = replace(PROB, transient=1, dt=0.01)
    opts = replace(OPTS, rtol=1e-12)
    orc = osolver.Oracle(prob, opts)
    N = orc.fine.N
    rng = np.random.default_rng(77)
    y = initial_state(prob, orc.fine, noise(N, 2))
    yn = y + 1e-4 * rng.standard_normal(N)
    ynm1 = yn + 1e-4 * rng.standard_normal(N)
    t = 0.37
    tr = dict(yn=yn, ynm1=ynm1, a=fem.bdf_coefficients(2), dt=prob.dt, t=t)
    r, J = orc.assemble(y, tr=tr)
    xs = osolver.direct_solve(J, -r)
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        s.set_state(_dev(y), _dev(yn), _dev(ynm1), t)
        rg = torch.empty(N, dtype=torch.float64, device="cuda")
        s.assemble(rg)
        assert np.max(np.abs(_host(rg) - r)) <= 1e-12 * np.max(np.abs(r))
        _rows_close(_csr(s, 1), J, 1e-12)
        dx = torch.empty(N, dtype=torch.float64, device="cuda")
        s.set_state(_dev(y), _dev(yn), _dev(ynm1), t)
        s.newton_step(dx)
        err = np.linalg.norm(_host(dx) - xs) / np.linalg.norm(xs)
        assert err <= 1e-10, err
    finally:
        s.close()


def test_3d_full_size_sampled_rows_bdf2():
    """The 3-level 3D box at full size (64 x 16 x 16 hexahedra, 908,422
    unknowns; the device assembles it in chunks of 1,024 elements per colour
    group): sampled node and pressure rows of the BDF2 Jacobian and residual
    against the oracle's element assembly of exactly the contributing
    elements, within 1e-12 of each row's largest entry.  The sampled nodes
    and elements are spread over the whole mesh, so rows of many chunks are
    compared."""
    from paper_1709_05660_gb300 import fsi
    from paper_1709_05660_gb300.workloads import CONFIGS
    from oracle.mesh import build_level
    from tests.test_gpu_parity import _check_rows, _oracle_rows
    prob, opts = CONFIGS["box3d_l3_bdf2"]
    s = fsi.FSI(prob, opts, stream=torch.cuda.current_stream().cuda_stream)
    try:
        N = int(s.N[-1])
        lev = build_level(prob, prob.levels - 1)
        assert N == lev.N
        y0 = initial_state(prob, lev, noise(N, 0))
        rng = np.random.default_rng(5)
        yp = y0 + 1e-4 * rng.standard_normal(N) * (~lev.dir_mask)
        ypp = yp + 1e-4 * rng.standard_normal(N) * (~lev.dir_mask)
        t = 3 * prob.dt
        s.set_state(_dev(y0), _dev(yp), _dev(ypp), t)
        r = torch.empty(N, dtype=torch.float64, device="cuda")
        s.assemble(r)
        Jg = _csr(s, prob.levels - 1)
        nodes = np.concatenate([rng.choice(lev.n_nodes, 40, replace=False),
                                np.nonzero(lev.node_class == 2)[0][::97]])
        elems_p = np.concatenate([rng.choice(lev.n_elem, 20, replace=False), np.nonzero(lev.elem_solid)[0][::41]])
        tr = dict(yn=yp, ynm1=ypp, a=fem.bdf_coefficients(2), dt=prob.dt, t=t)
        rows, rres = _oracle_rows(prob, lev, y0, nodes, elems_p, tr=tr)
        _check_rows(Jg, rows, 1e-12)
        rg = _host(r)
        rscale = max(1.0, np.max(np.abs(list(rres.values()))))
        for gi, v in rres.items():
            assert abs(rg[gi] - v) <= 1e-12 * rscale, gi
    finally:
        s.close()
