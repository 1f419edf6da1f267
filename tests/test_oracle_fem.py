"""Pins of the oracle's residual and exact Jacobian (CPU only).

* central finite differences of r(y) against the dual-number Jacobian;
* the structural zero blocks of the steady Jacobian listed in Sec. 3.1;
* manufactured-solution convergence rates of each physics on its own:
  Navier-Stokes (fluid), incompressible Neo-Hookean (solid) and the ALE
  mesh operator.  Q2 fields converge as h^3 in L2, the P1disc pressure as
  h^2; a dropped term, a wrong sign or a transposed index breaks the rate.
"""
from dataclasses import replace

import numpy as np
import pytest
import sympy as sy

from oracle import fem
from oracle.fem import GAUSS_W, GAUSS_X, q2_basis
from oracle.mesh import FLUID, IFACE, SOLID, build_level
from oracle.solver import direct_solve
from tests.oracle_cases import CHANNEL_2D, SMALL_3D, UNIT_FLUID, UNIT_SOLID, random_state


def _fd_check(prob, lev, seed, ndir=3, h=1e-6):
    y = random_state(lev, seed)
    r, J = fem.assemble(prob, lev, y)
    rng = np.random.default_rng(seed + 100)
    for _ in range(ndir):
        v = rng.standard_normal(lev.N)
        v[lev.N - (lev.N - lev.n_nodes * 2 * lev.dim):] *= 1.0
        rp = fem.residual_only(prob, lev, y + h * v)
        rm = fem.residual_only(prob, lev, y - h * v)
        fd = (rp - rm) / (2 * h)
        jv = J @ v
        err = np.linalg.norm(fd - jv) / np.linalg.norm(jv)
        assert err < 1e-6, err
    return y, J


def test_fd_jacobian_2d():
    lev = build_level(CHANNEL_2D, 0)
    y, J = _fd_check(CHANNEL_2D, lev, 1)
    # a few full columns at interface / solid / fluid / pressure unknowns
    nd = 4
    iface = np.nonzero(lev.node_class == IFACE)[0]
    cols = [iface[3] * nd + 0, iface[3] * nd + 3, np.nonzero(lev.node_class == SOLID)[0][0] * nd + 1,
            lev.n_nodes * nd + 5]
    h = 1e-6
    for c in cols:
        e = np.zeros(lev.N)
        e[c] = 1.0
        fd = (fem.residual_only(CHANNEL_2D, lev, y + h * e) - fem.residual_only(CHANNEL_2D, lev, y - h * e)) / (2 * h)
        col = J[:, c].toarray().ravel()
        scale = np.abs(col).max()
        assert np.abs(fd - col).max() <= 1e-6 * scale


def test_fd_jacobian_2d_harmonic_ale():
    prob = replace(CHANNEL_2D, ale_op=1)
    _fd_check(prob, build_level(prob, 0), 2, ndir=2)


def test_fd_jacobian_3d():
    _fd_check(SMALL_3D, build_level(SMALL_3D, 0), 3, ndir=2)


@pytest.mark.parametrize("prob", [CHANNEL_2D, SMALL_3D], ids=["2d", "3d"])
def test_steady_zero_blocks(prob):
    """Sec. 3.1: in the steady case the solid momentum does not depend on u,
    the solid kinematic rows not on d; the interface kinematic rows take
    nothing from fluid unknowns; ALE rows depend on d only; solid mass rows
    on d only.  These entries must be exactly 0.0."""
    lev = build_level(prob, 0)
    y = random_state(lev, 4)
    _, J = fem.assemble(prob, lev, y)
    J = J.tocsr()
    n, nd = lev.dim, 2 * lev.dim
    nn = lev.n_nodes * nd
    cls = lev.node_class
    free = ~lev.dir_mask
    col_node = np.arange(lev.N) // nd
    col_slot = np.arange(lev.N) % nd
    is_u_col = (np.arange(lev.N) < nn) & (col_slot >= n)
    is_d_col = (np.arange(lev.N) < nn) & (col_slot < n)
    is_p_col = np.arange(lev.N) >= nn
    fluid_col = (np.arange(lev.N) < nn) & (cls[np.minimum(col_node, lev.n_nodes - 1)] == FLUID)
    checked = 0
    for node in range(lev.n_nodes):
        for s in range(nd):
            row = node * nd + s
            if not free[row]:
                continue
            a, b = J.indptr[row], J.indptr[row + 1]
            c = J.indices[a:b]
            v = J.data[a:b]
            if cls[node] == SOLID and s < n:          # S rows: no u
                assert np.all(v[is_u_col[c]] == 0.0)
            if cls[node] != FLUID and s >= n:          # K rows: no d, no p, no fluid unknowns
                assert np.all(v[is_d_col[c]] == 0.0)
                assert np.all(v[is_p_col[c]] == 0.0)
                assert np.all(v[fluid_col[c]] == 0.0)
            if cls[node] == FLUID and s < n:           # A rows: d only
                assert np.all(v[~is_d_col[c]] == 0.0)
            if cls[node] == IFACE and s < n:           # I rows: no u of pure solid nodes
                solid_u = is_u_col[c] & (cls[np.minimum(col_node[c], lev.n_nodes - 1)] == SOLID)
                assert np.all(v[solid_u] == 0.0)
            checked += 1
    for e in np.nonzero(lev.elem_solid)[0]:             # V rows: d only
        for k in range(n + 1):
            row = nn + e * (n + 1) + k
            a, b = J.indptr[row], J.indptr[row + 1]
            assert np.all(J.data[a:b][~is_d_col[J.indices[a:b]]] == 0.0)
    assert checked > 0


# ----------------------------------------------------------------------------
# manufactured solutions
# ----------------------------------------------------------------------------

X, Y = sy.symbols("x y")


def _lambdify_vec(exprs):
    fs = [sy.lambdify((X, Y), e, "numpy", cse=True) for e in exprs]

    def f(xy):
        out = np.zeros((xy.shape[0], len(fs)))
        for i, g in enumerate(fs):
            out[:, i] = np.broadcast_to(g(xy[:, 0], xy[:, 1]), xy.shape[0])
        return out
    return f


def _l2_errors(lev, y, exact_d, exact_u, exact_p):
    """L2 errors of d, u (Q2) and p (P1disc, mean-free difference)."""
    nd, n = 4, 2
    ed = lev.elem_dofs
    err = {"d": 0.0, "u": 0.0}
    pdiff, pw = [], []
    for qx in range(3):
        for qy in range(3):
            xi = (GAUSS_X[qx], GAUSS_X[qy])
            w = GAUSS_W[qx] * GAUSS_W[qy] * np.prod(lev.elem_h, axis=1) / 4
            N, _ = q2_basis(2, xi)
            xq = lev.elem_lo + (np.array(xi)[None, :] + 1) * 0.5 * lev.elem_h
            ye = y[ed]
            for key, off, ex in (("d", 0, exact_d), ("u", n, exact_u)):
                val = np.stack([ye[:, np.arange(9) * nd + off + c] @ N for c in range(n)], axis=1)
                err[key] += np.sum(w * np.sum((val - ex(xq)) ** 2, axis=1))
            ph = ye[:, nd * 9:] @ np.array((1.0,) + xi)
            pdiff.append(ph - exact_p(xq)[:, 0])
            pw.append(w)
    pdiff = np.concatenate(pdiff)
    pw = np.concatenate(pw)
    mean = np.sum(pdiff * pw) / np.sum(pw)
    err["p"] = np.sum(pw * (pdiff - mean) ** 2)
    return {k: np.sqrt(v) for k, v in err.items()}


def _newton_direct(prob, lev, y, source, fix_pressure=False, steps=12):
    for _ in range(steps):
        r, J = fem.assemble(prob, lev, y, source)
        if fix_pressure:       # remove the constant-pressure kernel (pure-Dirichlet solid)
            J = J.tolil()
            p0 = lev.n_nodes * 4
            J.rows[p0] = [p0]
            J.data[p0] = [1.0]
            J = J.tocsr()
            r[p0] = 0.0
        dy = direct_solve(J, -r)
        y = y + dy
        if np.linalg.norm(dy) < 1e-11 * max(1.0, np.linalg.norm(y)):
            break
    return y


def _rates(prob, exact, source, fix_pressure=False, levels=(1, 2, 3)):
    ed_, eu_, ep_ = exact
    errs = []
    for l in levels:
        lev = build_level(prob, l)
        nd = 4
        y = np.zeros(lev.N)
        xyz = lev.node_xyz
        dex, uex = ed_(xyz), eu_(xyz)
        # Dirichlet data from the exact solution
        lev.dir_val[:] = 0.0
        for c in range(2):
            lev.dir_val[np.arange(lev.n_nodes) * nd + c] = dex[:, c]
            lev.dir_val[np.arange(lev.n_nodes) * nd + 2 + c] = uex[:, c]
        y[lev.dir_mask] = lev.dir_val[lev.dir_mask]
        y = _newton_direct(prob, lev, y, source, fix_pressure)
        errs.append(_l2_errors(lev, y, ed_, eu_, ep_))
    rates = {}
    if len(errs) > 1:
        rates = {k: np.log2(errs[-2][k] / errs[-1][k]) for k in errs[0] if errs[-1][k] > 1e-13}
    return errs, rates


def test_mms_navier_stokes():
    """Steady Navier-Stokes on a fixed mesh: traction-free outflow at x = 1."""
    rho, mu = UNIT_FLUID.rho_f, UNIT_FLUID.mu_f
    psi = (X - 1) ** 3 * sy.sin(sy.pi * Y)
    u = [sy.diff(psi, Y), -sy.diff(psi, X)]
    p = (X - 1) * sy.cos(sy.pi * Y) * 3
    grad = [[sy.diff(u[i], v) for v in (X, Y)] for i in range(2)]
    f = []
    for i in range(2):
        conv = sum(grad[i][j] * u[j] for j in range(2))
        lap = sum(sy.diff(u[i], v, 2) for v in (X, Y))
        f.append(sy.simplify(conv - mu / rho * lap + sy.diff(p, (X, Y)[i]) / rho))
    fm = _lambdify_vec(f)
    src = lambda xq: (fm(xq), np.zeros(len(xq)), None)
    ex = (_lambdify_vec([sy.Integer(0), sy.Integer(0)]), _lambdify_vec(u), _lambdify_vec([p]))
    errs, rates = _rates(UNIT_FLUID, ex, src)
    assert errs[-1]["d"] < 1e-12
    assert rates["u"] > 2.7, (errs, rates)
    assert rates["p"] > 1.8, (errs, rates)


def test_mms_neo_hookean_solid():
    """Incompressible Neo-Hookean (sigma = -p I + 2 C1 B): -div(J sigma F^{-T}) = rho f,
    J - 1 = g, steady kinematic u = 0."""
    mu = UNIT_SOLID.mu_s
    d = [sy.Rational(1, 20) * sy.sin(sy.pi * X) * sy.sin(sy.pi * Y),
         sy.Rational(1, 10) * X * Y * (1 - X) * (1 + Y)]
    p = sy.cos(sy.pi * X) * sy.cos(sy.pi * Y)
    F = sy.Matrix([[1 + sy.diff(d[0], X), sy.diff(d[0], Y)], [sy.diff(d[1], X), 1 + sy.diff(d[1], Y)]])
    J = F.det()
    P = -p * J * F.inv().T + mu * J * F
    f = [-(sy.diff(P[i, 0], X) + sy.diff(P[i, 1], Y)) / UNIT_SOLID.rho_s for i in range(2)]
    fm = _lambdify_vec(f)
    gm = _lambdify_vec([J - 1])
    src = lambda xq: (fm(xq), gm(xq)[:, 0], None)
    ex = (_lambdify_vec(d), _lambdify_vec([sy.Integer(0), sy.Integer(0)]), _lambdify_vec([p]))
    errs, rates = _rates(UNIT_SOLID, ex, src, fix_pressure=True)
    assert errs[-1]["u"] < 1e-12
    assert rates["d"] > 2.7, (errs, rates)
    assert rates["p"] > 1.8, (errs, rates)


def test_mms_ale_operator():
    """Mesh equation -div(k (grad d + grad d^T)) = g, k = 1/V_el, with u = p = 0."""
    d = [sy.sin(sy.pi * X) * Y * Y * sy.Rational(1, 10), sy.cos(sy.pi * Y) * X * sy.Rational(1, 10)]
    g = []
    for i in range(2):
        s = 0
        for j, v in enumerate((X, Y)):
            s += sy.diff(sy.diff(d[i], v) + sy.diff(d[j], (X, Y)[i]), v)
        g.append(-s)
    gf = _lambdify_vec(g)
    ex = (_lambdify_vec(d), _lambdify_vec([sy.Integer(0)] * 2), _lambdify_vec([sy.Integer(0)]))
    errs = []
    for l in (1, 2, 3):
        h = 0.5 / 2 ** l
        k = 1.0 / (h * h)
        src = lambda xq, k=k: (np.zeros((len(xq), 2)), np.zeros(len(xq)), k * gf(xq))
        e, _ = _rates(UNIT_FLUID, ex, src, levels=(l,))
        errs.append(e[0])
    rate = np.log2(errs[-2]["d"] / errs[-1]["d"])
    assert rate > 2.7, errs
    assert errs[-1]["u"] < 1e-12


# ----------------------------------------------------------------------------
# transient (BDF) form
# ----------------------------------------------------------------------------

def _tr_state(lev, seed):
    rng = np.random.default_rng(seed)
    y = random_state(lev, seed)
    yn = y + 1e-3 * rng.standard_normal(lev.N)
    ynm1 = yn + 1e-3 * rng.standard_normal(lev.N)
    return y, yn, ynm1


@pytest.mark.parametrize("prob,order", [(CHANNEL_2D, 2), (CHANNEL_2D, 1), (SMALL_3D, 2)], ids=["2d-bdf2", "2d-bdf1", "3d-bdf2"])
def test_fd_jacobian_transient(prob, order):
    lev = build_level(prob, 0)
    y, yn, ynm1 = _tr_state(lev, 7)
    tr = dict(yn=yn, ynm1=ynm1, a=fem.bdf_coefficients(order), dt=0.01, t=0.13)
    r, J = fem.assemble(prob, lev, y, tr=tr)
    rng = np.random.default_rng(8)
    h = 1e-6
    for _ in range(2):
        v = rng.standard_normal(lev.N)
        fd = (fem.residual_only(prob, lev, y + h * v, tr=tr) - fem.residual_only(prob, lev, y - h * v, tr=tr)) / (2 * h)
        jv = J @ v
        assert np.linalg.norm(fd - jv) <= 1e-6 * np.linalg.norm(jv)


def test_transient_reduces_to_steady_for_constant_history():
    """y_n = y_{n-1} = y: every BDF derivative vanishes (a0 + a1 + a2 = 0) and
    the mesh velocity is zero, so the transient residual is the steady one
    (alpha(1/4) = 1 keeps the inflow data equal)."""
    prob = CHANNEL_2D
    lev = build_level(prob, 0)
    y = random_state(lev, 9)
    r0, J0 = fem.assemble(prob, lev, y)
    tr = dict(yn=y.copy(), ynm1=y.copy(), a=fem.bdf_coefficients(2), dt=0.01, t=0.25)
    r1, _ = fem.assemble(prob, lev, y, tr=tr)
    assert np.max(np.abs(r1 - r0)) <= 1e-12 * np.max(np.abs(r0))


def test_transient_kinematic_rows_vanish_for_consistent_velocity():
    """Solid kinematic rows: with d linear in time and nodal u equal to its
    BDF derivative, (u - d_t, psi) = 0 exactly (BDF1 and BDF2)."""
    prob = CHANNEL_2D
    lev = build_level(prob, 0)
    rng = np.random.default_rng(10)
    nd, n = 4, 2
    dt = 0.02
    for order in (1, 2):
        y = np.zeros(lev.N)
        delta = np.zeros(lev.N)
        for c in range(n):
            delta[c:lev.n_nodes * nd:nd] = 1e-3 * rng.standard_normal(lev.n_nodes)
        y[:] = delta * 3
        yn, ynm1 = y - delta, y - 2 * delta
        for c in range(n):
            y[n + c:lev.n_nodes * nd:nd] = delta[c:lev.n_nodes * nd:nd] / dt
        tr = dict(yn=yn, ynm1=ynm1, a=fem.bdf_coefficients(order), dt=dt, t=0.0)
        r, _ = fem.assemble(prob, lev, y, tr=tr)
        kin_rows = [node * nd + n + c for node in np.nonzero(lev.node_class != FLUID)[0] for c in range(n)
                    if not lev.dir_mask[node * nd + n + c]]
        scale = np.max(np.abs(y[n:lev.n_nodes * nd:nd])) * np.max(lev.elem_h) ** 2
        assert np.max(np.abs(r[kin_rows])) <= 1e-12 * scale


# ----------------------------------------------------------------------------
# fluid terms on a deformed mesh (F != I)
# ----------------------------------------------------------------------------

def _quad_map():
    """A quadratic displacement d(x_hat) (exactly representable in Q2, so the
    discrete mesh equals the exact one), its gradient and det F.  F = I +
    grad_hat d is non-constant and non-symmetric."""
    def d(xh):
        x, y = xh[:, 0], xh[:, 1]
        return np.stack([0.12 * x * y + 0.05 * y * y, 0.1 * x * x - 0.07 * x * y], axis=1)

    def detF(xh):
        x, y = xh[:, 0], xh[:, 1]
        F = np.array([[1 + 0.12 * y, 0.12 * x + 0.1 * y], [0.2 * x - 0.07 * y, 1 - 0.07 * x]])
        return F[0, 0] * F[1, 1] - F[0, 1] * F[1, 0]
    return d, detF


def test_mms_navier_stokes_deformed_mesh():
    """Navier-Stokes on a fixed curved mesh x = x_hat + d(x_hat) (Sec. 2.1,
    2.3): the manufactured solution is a smooth field of the physical
    coordinates; every displacement unknown and every boundary velocity is a
    Dirichlet value.  The ALE form maps gradients by F^{-T} and weights by J,
    so a transposed F^{-1}, or J dropped from a term, converges to another
    field and breaks the rates (at d = 0 these factors are the identity)."""
    rho, mu = UNIT_FLUID.rho_f, UNIT_FLUID.mu_f
    psi = sy.sin(sy.pi * X) * sy.sin(sy.pi * Y) * sy.Rational(1, 2)
    u = [sy.diff(psi, Y), -sy.diff(psi, X)]
    p = sy.cos(sy.pi * X) * sy.sin(sy.pi * Y)
    grad = [[sy.diff(u[i], v) for v in (X, Y)] for i in range(2)]
    f = [sy.simplify(sum(grad[i][j] * u[j] for j in range(2)) - mu / rho * sum(sy.diff(u[i], v, 2) for v in (X, Y))
                     + sy.diff(p, (X, Y)[i]) / rho) for i in range(2)]
    fm_phys, u_phys, p_phys = _lambdify_vec(f), _lambdify_vec(u), _lambdify_vec([p])
    dmap, detF = _quad_map()
    to_phys = lambda xh: xh + dmap(xh)
    # the source callback integrates -(rho f, phi) over the reference element,
    # so the physical body force carries the Jacobian of the map
    src = lambda xh: (fm_phys(to_phys(xh)) * detF(xh)[:, None], np.zeros(len(xh)), None)
    ex_d = dmap
    ex_u = lambda xh: u_phys(to_phys(xh))
    ex_p = lambda xh: p_phys(to_phys(xh))
    errs = []
    for l in (1, 2, 3):
        lev = build_level(UNIT_FLUID, l)
        nd = 4
        xyz = lev.node_xyz
        bnd = np.zeros(lev.n_nodes, dtype=bool)
        for a in range(2):
            bnd |= np.isclose(xyz[:, a], 0.0) | np.isclose(xyz[:, a], 1.0)
        lev.dir_mask[:] = False
        for c in range(2):
            lev.dir_mask[np.arange(lev.n_nodes) * nd + c] = True            # the mesh is fixed
            lev.dir_mask[np.nonzero(bnd)[0] * nd + 2 + c] = True             # velocity on all walls
        dv, uv = ex_d(xyz), ex_u(xyz)
        lev.dir_val[:] = 0.0
        for c in range(2):
            lev.dir_val[np.arange(lev.n_nodes) * nd + c] = dv[:, c]
            lev.dir_val[np.arange(lev.n_nodes) * nd + 2 + c] = uv[:, c]
        y = np.zeros(lev.N)
        y[lev.dir_mask] = lev.dir_val[lev.dir_mask]
        y = _newton_direct(UNIT_FLUID, lev, y, src, fix_pressure=True)
        errs.append(_l2_errors(lev, y, ex_d, ex_u, ex_p))
    ru = np.log2(errs[-2]["u"] / errs[-1]["u"])
    rp = np.log2(errs[-2]["p"] / errs[-1]["p"])
    assert errs[-1]["d"] < 1e-12
    assert ru > 2.7, (errs, ru)
    assert rp > 1.8, (errs, rp)


# ----------------------------------------------------------------------------
# transient terms: inertia with J, and the mesh velocity in the convection
# ----------------------------------------------------------------------------

SIMPSON = np.array([1.0, 4.0, 1.0]) / 6.0     # integrals of the 1D Q2 basis over a unit cell


def _affine_state(lev, A, rng, p_amp=30.0):
    """d = (A - I) x_hat at every node (F = A), random pressures."""
    nd, n = 2 * lev.dim, lev.dim
    y = np.zeros(lev.N)
    dvals = lev.node_xyz @ (A - np.eye(n)).T
    for c in range(n):
        y[c:lev.n_nodes * nd:nd] = dvals[:, c]
    y[lev.n_nodes * nd:] = p_amp * rng.standard_normal(lev.N - lev.n_nodes * nd)
    return y


def _basis_integrals(lev):
    """(E, 3^dim): exact integral of each element's Q2 basis functions over
    the (undeformed) element, by the product of 1D Simpson weights."""
    nloc = 3 ** lev.dim
    w = np.ones((lev.n_elem, nloc))
    for a in range(nloc):
        for d in range(lev.dim):
            w[:, a] *= SIMPSON[(a // 3 ** d) % 3] * lev.elem_h[:, d]
    return w


_A2 = np.array([[1.45, 0.2], [-0.15, 0.92]])
_A3 = np.array([[1.3, 0.1, -0.05], [0.08, 1.1, 0.12], [-0.1, 0.05, 0.95]])


@pytest.mark.parametrize("prob,order", [(CHANNEL_2D, 1), (CHANNEL_2D, 2), (SMALL_3D, 2)],
                         ids=["2d-bdf1", "2d-bdf2", "3d-bdf2"])
def test_transient_inertia_closed_form(prob, order):
    """Uniform acceleration on an affinely deformed mesh (F = A constant):
    nodal velocities linear in time, u_t = c, grad u = 0, displacement
    constant in time (w = 0).  The transient residual minus the steady one is
    then the inertia term alone: rho J c_i times the integral of the test
    function, with J = det A, fluid rows weighted by rho_f and solid rows by
    rho_s (interface rows both); every other row is unchanged.  The basis
    integrals come from Simpson's weights, not from the oracle's quadrature."""
    prob = replace(prob, rho_s=700.0)
    lev = build_level(prob, 0)
    n, nd = lev.dim, 2 * lev.dim
    A = _A2 if n == 2 else _A3
    rng = np.random.default_rng(21)
    y = _affine_state(lev, A, rng)
    U0 = rng.standard_normal(n)
    c = rng.standard_normal(n) * 3.0
    dt = 0.02
    hist = []
    for k in (0, 1, 2):
        yk = y.copy()
        for i in range(n):
            yk[n + i:lev.n_nodes * nd:nd] = U0[i] - k * c[i] * dt
        hist.append(yk)
    tr = dict(yn=hist[1], ynm1=hist[2], a=fem.bdf_coefficients(order), dt=dt, t=0.25)
    r_tr = fem.residual_only(prob, lev, hist[0], tr=tr)
    r_st = fem.residual_only(prob, lev, hist[0])
    want = np.zeros(lev.N)
    wint = _basis_integrals(lev)
    detA = np.linalg.det(A)
    for e in range(lev.n_elem):
        solid = bool(lev.elem_solid[e])
        for a, node in enumerate(lev.elem_nodes[e]):
            cls = lev.node_class[node]
            slot0 = 0 if (solid or cls == IFACE) else n      # momentum rows: d-rows of solid / interface nodes
            rho = prob.rho_s if solid else prob.rho_f
            for i in range(n):
                want[node * nd + slot0 + i] += rho * detA * c[i] * wint[e, a]
    free = ~lev.dir_mask
    got = (r_tr - r_st)[free]
    scale = np.max(np.abs(want))
    assert scale > 0
    assert np.max(np.abs(got - want[free])) <= 1e-11 * scale


@pytest.mark.parametrize("prob,order", [(CHANNEL_2D, 1), (CHANNEL_2D, 2), (SMALL_3D, 2)],
                         ids=["2d-bdf1", "2d-bdf2", "3d-bdf2"])
def test_transient_galilean_mesh_velocity(prob, order):
    """Galilean invariance of the ALE form: translate an (affinely deformed)
    state rigidly with constant velocity V, i.e. displacement d + V t and
    velocity u + V at every node.  The BDF mesh velocity is then exactly
    w = V and u_t = 0, so the convective velocity u + V - w, the solid
    kinematic velocity u + V - d_t and every gradient are those of the
    untranslated steady state: all free rows of the transient residual equal
    the steady residual of (d, u, p).  A wrong sign of w, w missing from the
    convection or d_t missing from the kinematic rows breaks the identity."""
    lev = build_level(prob, 0)
    n, nd = lev.dim, 2 * lev.dim
    A = _A2 if n == 2 else _A3
    rng = np.random.default_rng(22)
    base = _affine_state(lev, A, rng)
    for i in range(n):
        base[n + i:lev.n_nodes * nd:nd] = 0.4 * rng.standard_normal(lev.n_nodes)
    V = rng.standard_normal(n) * 0.7
    dt, t1 = 0.03, 0.25
    hist = []
    for k in (0, 1, 2):
        yk = base.copy()
        for i in range(n):
            yk[i:lev.n_nodes * nd:nd] += V[i] * (t1 - k * dt)
            yk[n + i:lev.n_nodes * nd:nd] += V[i]
        hist.append(yk)
    tr = dict(yn=hist[1], ynm1=hist[2], a=fem.bdf_coefficients(order), dt=dt, t=t1)
    r_tr = fem.residual_only(prob, lev, hist[0], tr=tr)
    r_st = fem.residual_only(prob, lev, base)
    free = ~lev.dir_mask
    scale = np.max(np.abs(r_st[free]))
    assert np.max(np.abs(r_tr[free] - r_st[free])) <= 1e-11 * scale
    # the same translation without the mesh moving along (w = 0) is not invariant
    for k in range(3):
        for i in range(n):
            hist[k][i:lev.n_nodes * nd:nd] -= V[i] * (t1 - k * dt)
    r_fixed = fem.residual_only(prob, lev, hist[0], tr=dict(tr, yn=hist[1], ynm1=hist[2]))
    assert np.max(np.abs(r_fixed[free] - r_st[free])) > 1e-6 * scale


@pytest.mark.parametrize("prob", [CHANNEL_2D, SMALL_3D], ids=["2d", "3d"])
def test_mass_rows_affine_closed_form(prob):
    """Mass rows on an affinely deformed mesh (x = A x_hat, F = A) with a
    velocity linear in the physical coordinates, u = B x + b (exactly a Q2
    field).  A fluid element's rows are the integrals of div u times the
    P1disc test functions over the deformed element: tr(B) |det A| |e| for
    q = 1 and 0 for q = xi, eta(, zeta) (odd about the element centre); a
    solid element's rows are the integrals of J - 1: (det A - 1) |e| and 0."""
    lev = build_level(prob, 0)
    n, nd = lev.dim, 2 * lev.dim
    A = _A2 if n == 2 else _A3
    rng = np.random.default_rng(23)
    y = _affine_state(lev, A, rng)
    Bm = rng.standard_normal((n, n))
    bv = rng.standard_normal(n)
    uval = (lev.node_xyz @ A.T) @ Bm.T + bv
    for i in range(n):
        y[n + i:lev.n_nodes * nd:nd] = uval[:, i]
    r = fem.residual_only(prob, lev, y)
    vol = np.prod(lev.elem_h, axis=1)
    detA = np.linalg.det(A)
    p0 = lev.n_nodes * nd
    want = np.zeros((lev.n_elem, n + 1))
    want[:, 0] = np.where(lev.elem_solid, (detA - 1.0) * vol, np.trace(Bm) * detA * vol)
    got = r[p0:].reshape(lev.n_elem, n + 1)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


# ----------------------------------------------------------------------------
# Mooney-Rivlin solid (Sec. 2.2): sigma = -p I + 2 C1 B - 2 C2 B^{-1}
# ----------------------------------------------------------------------------

def test_mms_mooney_rivlin_solid():
    """Incompressible Mooney-Rivlin with C2 = 0.3, C1 = mu_s / 2 - C2:
    -div(J sigma F^{-T}) = rho f, J - 1 = g.  A wrong sign or a transposed
    factor of the B^{-1} term converges to another field and breaks the
    rates."""
    c2 = 0.3
    prob = replace(UNIT_SOLID, mr_c2=c2)
    mu = prob.mu_s
    d = [sy.Rational(1, 20) * sy.sin(sy.pi * X) * sy.sin(sy.pi * Y),
         sy.Rational(1, 10) * X * Y * (1 - X) * (1 + Y)]
    p = sy.cos(sy.pi * X) * sy.cos(sy.pi * Y)
    F = sy.Matrix([[1 + sy.diff(d[0], X), sy.diff(d[0], Y)], [sy.diff(d[1], X), 1 + sy.diff(d[1], Y)]])
    J = F.det()
    Bm = F * F.T
    adj = lambda M: sy.Matrix([[M[1, 1], -M[0, 1]], [-M[1, 0], M[0, 0]]])   # det(B) = J^2
    sigma = -p * sy.eye(2) + (mu - 2 * c2) * Bm - 2 * c2 * adj(Bm) / J ** 2
    P = J * sigma * adj(F).T / J
    f = [-(sy.diff(P[i, 0], X) + sy.diff(P[i, 1], Y)) / prob.rho_s for i in range(2)]
    fm = _lambdify_vec(f)
    gm = _lambdify_vec([J - 1])
    src = lambda xq: (fm(xq), gm(xq)[:, 0], None)
    ex = (_lambdify_vec(d), _lambdify_vec([sy.Integer(0), sy.Integer(0)]), _lambdify_vec([p]))
    errs, rates = _rates(prob, ex, src, fix_pressure=True)
    assert errs[-1]["u"] < 1e-12
    assert rates["d"] > 2.7, (errs, rates)
    assert rates["p"] > 1.8, (errs, rates)


@pytest.mark.parametrize("dim", [2, 3])
def test_mooney_rivlin_rigid_rotation_is_stress_free(dim):
    """A rigid rotation d = (Q - I) x_hat has B = I, so with the element
    pressures at 2 C1 - 2 C2 = mu_s - 4 C2 the Mooney-Rivlin stress vanishes:
    every free row of an all-solid mesh is zero (momentum, J - 1 = 0, u = 0),
    including the displacement rows of a traction-free face (x = max, its
    displacements freed here).  A pressure balancing 2 C1 + 2 C2 instead (the
    C2 term with the other sign) leaves a hydrostatic stress whose traction
    on that face is nonzero."""
    c2 = 0.21
    if dim == 2:
        prob = replace(UNIT_SOLID, mr_c2=c2)
        th = 0.4
        Q = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    else:
        prob = replace(SMALL_3D, flap_lo=(-1.0, -1.0, -1.0), flap_hi=(2.0, 2.0, 2.0), mr_c2=c2 * 1e5)
        a, b = 0.3, -0.5
        Qx = np.array([[1, 0, 0], [0, np.cos(a), -np.sin(a)], [0, np.sin(a), np.cos(a)]])
        Qz = np.array([[np.cos(b), -np.sin(b), 0], [np.sin(b), np.cos(b), 0], [0, 0, 1]])
        Q = Qz @ Qx
    lev = build_level(prob, 1 if dim == 2 else 0)
    assert np.all(lev.elem_solid)
    n, nd = lev.dim, 2 * lev.dim
    right = np.nonzero(np.isclose(lev.node_xyz[:, 0], lev.node_xyz[:, 0].max()))[0]
    for c in range(n):
        lev.dir_mask[right * nd + c] = False
    y = np.zeros(lev.N)
    dv = lev.node_xyz @ (Q - np.eye(n)).T
    for c in range(n):
        y[c:lev.n_nodes * nd:nd] = dv[:, c]
    p0 = lev.n_nodes * nd
    y[p0::n + 1] = prob.mu_s - 4.0 * prob.mr_c2
    r = fem.residual_only(prob, lev, y)
    free = ~lev.dir_mask
    scale = prob.mu_s * np.max(lev.elem_h) ** (dim - 1)
    assert np.max(np.abs(r[free])) <= 1e-10 * scale
    y[p0::n + 1] = prob.mu_s            # a pressure that balances 2 C1 + 2 C2 instead
    r = fem.residual_only(prob, lev, y)
    assert np.max(np.abs(r[free])) > 1e-3 * prob.mr_c2 * np.min(lev.elem_h) ** (dim - 1)


@pytest.mark.parametrize("prob", [replace(CHANNEL_2D, mr_c2=8e4), replace(SMALL_3D, mr_c2=6e4)], ids=["2d", "3d"])
def test_fd_jacobian_mooney_rivlin(prob):
    _fd_check(prob, build_level(prob, 0), 31, ndir=2)


# ----------------------------------------------------------------------------
# Crank-Nicolson form of Sec. 2.5 (conservative ALE identity of Sec. 2.3)
# ----------------------------------------------------------------------------

def _cn(yn, dt, t=0.25):
    return dict(scheme="cn", yn=yn, dt=dt, t=t)


@pytest.mark.parametrize("prob", [replace(CHANNEL_2D, mr_c2=5e4), SMALL_3D], ids=["2d", "3d"])
def test_fd_jacobian_crank_nicolson(prob):
    lev = build_level(prob, 0)
    y, yn, _ = _tr_state(lev, 17)
    tr = _cn(yn, 0.02)
    r, J = fem.assemble(prob, lev, y, tr=tr)
    rng = np.random.default_rng(18)
    h = 1e-6
    for _ in range(2):
        v = rng.standard_normal(lev.N)
        fd = (fem.residual_only(prob, lev, y + h * v, tr=tr) - fem.residual_only(prob, lev, y - h * v, tr=tr)) / (2 * h)
        jv = J @ v
        assert np.linalg.norm(fd - jv) <= 1e-6 * np.linalg.norm(jv)


@pytest.mark.parametrize("prob", [CHANNEL_2D, SMALL_3D], ids=["2d", "3d"])
def test_cn_galilean_invariance(prob):
    """Rigid translation with velocity V between t_n and t_{n+1} (d + V t,
    u + V at both levels): the conservative inertia vanishes, div w = 0, the
    convective velocity u + V - w and the kinematic velocity (u + V) - w are
    those of the untranslated state, and both stress halves coincide, so every
    free row equals the steady residual of (d, u, p)."""
    lev = build_level(prob, 0)
    n, nd = lev.dim, 2 * lev.dim
    A = _A2 if n == 2 else _A3
    rng = np.random.default_rng(24)
    base = _affine_state(lev, A, rng)
    for i in range(n):
        base[n + i:lev.n_nodes * nd:nd] = 0.4 * rng.standard_normal(lev.n_nodes)
    V = rng.standard_normal(n) * 0.7
    dt, t1 = 0.03, 0.25
    ys = []
    for k in (0, 1):
        yk = base.copy()
        for i in range(n):
            yk[i:lev.n_nodes * nd:nd] += V[i] * (t1 - k * dt)
            yk[n + i:lev.n_nodes * nd:nd] += V[i]
        ys.append(yk)
    r_cn = fem.residual_only(prob, lev, ys[0], tr=_cn(ys[1], dt, t1))
    r_st = fem.residual_only(prob, lev, base)
    free = ~lev.dir_mask
    scale = np.max(np.abs(r_st[free]))
    assert np.max(np.abs(r_cn[free] - r_st[free])) <= 1e-11 * scale


@pytest.mark.parametrize("prob", [CHANNEL_2D, SMALL_3D], ids=["2d", "3d"])
def test_cn_uniform_acceleration_closed_form(prob):
    """Affinely deformed mesh at rest (w = 0, F = A), velocities uniform in
    space with u_{n+1} - u_n = c dt, same pressures at both levels: relative
    to the steady residual of the new state, the momentum rows gain
    rho J c times the integral of the test function (rho_f on fluid, rho_s on
    solid elements) and the solid kinematic rows, (u_{n+1} + u_n)/2 - w
    instead of u_{n+1}, lose c dt / 2 times it; nothing else changes."""
    prob = replace(prob, rho_s=700.0)
    lev = build_level(prob, 0)
    n, nd = lev.dim, 2 * lev.dim
    A = _A2 if n == 2 else _A3
    rng = np.random.default_rng(25)
    y = _affine_state(lev, A, rng)
    U0 = rng.standard_normal(n)
    c = rng.standard_normal(n) * 3.0
    dt = 0.02
    y1, y0 = y.copy(), y.copy()
    for i in range(n):
        y1[n + i:lev.n_nodes * nd:nd] = U0[i]
        y0[n + i:lev.n_nodes * nd:nd] = U0[i] - c[i] * dt
    r_cn = fem.residual_only(prob, lev, y1, tr=_cn(y0, dt))
    r_st = fem.residual_only(prob, lev, y1)
    want = np.zeros(lev.N)
    wint = _basis_integrals(lev)
    detA = np.linalg.det(A)
    for e in range(lev.n_elem):
        solid = bool(lev.elem_solid[e])
        for a, node in enumerate(lev.elem_nodes[e]):
            cls = lev.node_class[node]
            slot0 = 0 if (solid or cls == IFACE) else n
            rho = prob.rho_s if solid else prob.rho_f
            for i in range(n):
                want[node * nd + slot0 + i] += rho * detA * c[i] * wint[e, a]
                if solid:
                    want[node * nd + n + i] += -0.5 * c[i] * dt * wint[e, a]
    free = ~lev.dir_mask
    got = (r_cn - r_st)[free]
    assert np.max(np.abs(got - want[free])) <= 1e-11 * np.max(np.abs(want))


def test_cn_geometric_conservation_2d():
    """Discrete geometric conservation in 2D: a uniform velocity on a mesh
    moving affinely (d = (A(t) - I) x_hat with A linear in t, so J is
    quadratic and J div w linear in t) leaves every free fluid momentum row
    at zero (p = 0): the conservative difference of J u over the step equals
    the trapezoidal average of J (div w) u exactly.  A wrong sign or weight
    of the -(div w) u terms breaks it."""
    lev = build_level(UNIT_FLUID, 1)
    n, nd = 2, 4
    B = np.array([[0.8, -0.3], [0.5, 0.6]])
    dt, t1 = 0.05, 0.4
    U = np.array([0.7, -0.4])
    ys = []
    for t in (t1, t1 - dt):
        yk = np.zeros(lev.N)
        dv = lev.node_xyz @ (t * B).T
        for i in range(n):
            yk[i:lev.n_nodes * nd:nd] = dv[:, i]
            yk[n + i:lev.n_nodes * nd:nd] = U[i]
        ys.append(yk)
    r = fem.residual_only(UNIT_FLUID, lev, ys[0], tr=_cn(ys[1], dt, 0.25))
    rows = [node * nd + n + i for node in range(lev.n_nodes) for i in range(n) if not lev.dir_mask[node * nd + n + i]]
    scale = UNIT_FLUID.rho_f * np.max(np.abs(U)) * np.max(lev.elem_h) ** 2 / dt
    assert np.max(np.abs(r[rows])) <= 1e-12 * scale


@pytest.mark.parametrize("scheme,rate", [("cn", 2.0), ("bdf1", 1.0), ("bdf2", 2.0)])
def test_temporal_rate_solid_shear_oscillation(scheme, rate):
    """A manufactured solution in time: an incompressible Neo-Hookean block in
    homogeneous simple shear d = s(t) (y, 0), u = s'(t) (y, 0), p = mu_s
    (stress constant in space, J = 1), driven by the body force
    f = s''(t) (y, 0) with all boundary values prescribed.  The space
    discretisation is exact, so the error at T is the time discretisation's:
    second order for Crank-Nicolson (trapezoidal inertia and kinematics with
    the averaged force) and BDF2 (BDF1 start), first order for BDF1."""
    prob = UNIT_SOLID
    om = 2.0 * np.pi
    s = lambda t: 0.05 * np.sin(om * t)
    s1 = lambda t: 0.05 * om * np.cos(om * t)
    s2 = lambda t: -0.05 * om * om * np.sin(om * t)
    T = 0.4
    errs = []
    for nsteps in (16, 32, 64):
        lev = build_level(prob, 1)
        nd = 4
        dt = T / nsteps
        yy = lev.node_xyz[:, 1]
        p0 = lev.n_nodes * nd

        def exact(t):
            y = np.zeros(lev.N)
            y[0:p0:nd] = s(t) * yy
            y[2:p0:nd] = s1(t) * yy
            y[p0::3] = prob.mu_s
            return y

        hist = [exact(0.0)]
        for k in range(1, nsteps + 1):
            t = k * dt
            ex = exact(t)
            lev.dir_val[:] = ex
            if scheme == "cn":
                tr = _cn(hist[-1], dt)
                fsrc = lambda xq, t=t: 0.5 * (s2(t) + s2(t - dt)) * xq[:, 1]
            else:
                order = 1 if (scheme == "bdf1" or k == 1) else 2
                tr = dict(yn=hist[-1], ynm1=hist[-2] if order == 2 else hist[-1],
                          a=fem.bdf_coefficients(order), dt=dt, t=0.25)
                fsrc = lambda xq, t=t: s2(t) * xq[:, 1]
            src = lambda xq, f=fsrc: (np.stack([f(xq), np.zeros(len(xq))], axis=1), np.zeros(len(xq)), None)
            y = hist[-1].copy()
            y[lev.dir_mask] = ex[lev.dir_mask]
            for _ in range(8):
                r, J = fem.assemble(prob, lev, y, src, tr=tr)
                J = J.tolil()
                J.rows[p0] = [p0]
                J.data[p0] = [1.0]
                J = J.tocsr()
                r[p0] = y[p0] - prob.mu_s
                dy = direct_solve(J, -r)
                y = y + dy
                if np.linalg.norm(dy) < 1e-13 * np.linalg.norm(y):
                    break
            hist.append(y)
        e = hist[-1] - exact(T)
        errs.append(np.max(np.abs(e[0:lev.n_nodes * nd:nd])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > rate - 0.15, (errs, rates)
    assert rates[-1] < rate + 0.5, (errs, rates)
