"""Pins of the oracle's multigrid / Schwarz / Krylov parts (CPU only).

* prolongation reproduces coarse Q2 and P1disc fields exactly, checked by an
  independent evaluation in physical coordinates (natural injection, Sec. 3.2);
* restriction = transpose of prolongation except the interface rule of
  Sec. 3.2, entry by entry;
* Galerkin coarse operator = rediscretisation on the coarse mesh for the
  Jacobian at y = 0, where every physics is a constant-coefficient bilinear
  form integrated exactly (ALE rows scale with k = 1/V_el, i.e. 2^dim);
* restricted additive Schwarz: one subdomain + omega = 1 converges in one
  Richardson step; two subdomains match the dense formula of Sec. 3.3;
* FGMRES: identity preconditioner on a diagonal system converges in at most
  n steps; with the V-cycle it reproduces the sparse direct solve.
"""
from dataclasses import replace

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fem, solver
from oracle.mesh import FLUID, IFACE, SOLID, Patch, build_level, initial_state
from paper_1709_05660_gb300.workloads import CONFIGS, SolverOpts, noise
from tests.oracle_cases import CHANNEL_2D, SMALL_3D, random_state


def _lagrange_phys(nodes, x):
    """1D quadratic Lagrange basis through 3 physical nodes, evaluated at x."""
    out = []
    for m in range(3):
        v = np.ones_like(x)
        for k in range(3):
            if k != m:
                v = v * (x - nodes[k]) / (nodes[m] - nodes[k])
        out.append(v)
    return out


@pytest.mark.parametrize("prob", [CHANNEL_2D, replace(SMALL_3D, levels=2)], ids=["2d", "3d"])
def test_prolongation_reproduces_coarse_fields(prob):
    coarse, fine = build_level(prob, 0), build_level(prob, 1)
    P = solver.prolongation(coarse, fine)
    rng = np.random.default_rng(0)
    vc = rng.standard_normal(coarse.N)
    vf = P @ vc
    dim, nd = prob.dim, 2 * prob.dim
    # nodal fields: evaluate coarse interpolant at every fine node in physical coordinates
    for f in range(fine.n_nodes):
        x = fine.node_xyz[f]
        cell = [min(np.searchsorted(coarse.verts[d], x[d], side="right") - 1, coarse.cells[d] - 1)
                for d in range(dim)]
        w1d = []
        for d in range(dim):
            nodes = coarse.coords[d][2 * cell[d]: 2 * cell[d] + 3]
            w1d.append(_lagrange_phys(nodes, np.array(x[d])))
        for s in range(nd):
            val = 0.0
            for a in range(3 ** dim):
                idx = [(a // 3 ** d) % 3 for d in range(dim)]
                wgt = np.prod([w1d[d][idx[d]] for d in range(dim)])
                cn = 0
                stride = 1
                for d in range(dim):
                    cn += (2 * cell[d] + idx[d]) * stride
                    stride *= coarse.nodes_ax[d]
                val += wgt * vc[cn * nd + s]
            assert abs(vf[f * nd + s] - val) <= 1e-13 * (1 + abs(val))
    # pressures: coarse linear function vs fine linear function at fine-element corners
    for ef in range(fine.n_elem):
        lo, h = fine.elem_lo[ef], fine.elem_h[ef]
        cen = lo + 0.5 * h
        ec = 0
        stride = 1
        clo = np.zeros(dim)
        ch = np.zeros(dim)
        for d in range(dim):
            ci = np.searchsorted(coarse.verts[d], cen[d]) - 1
            ec += ci * stride
            stride *= coarse.cells[d]
            clo[d], ch[d] = coarse.verts[d][ci], coarse.verts[d][ci + 1] - coarse.verts[d][ci]
        pc = vc[coarse.n_nodes * nd + ec * (dim + 1):][: dim + 1]
        pf = vf[fine.n_nodes * nd + ef * (dim + 1):][: dim + 1]
        for corner in range(2 ** dim):
            xp = lo + np.array([(corner >> d) & 1 for d in range(dim)]) * h
            xi_c = 2 * (xp - clo) / ch - 1
            xi_f = 2 * (xp - lo) / h - 1
            assert abs(pc[0] + pc[1:] @ xi_c - (pf[0] + pf[1:] @ xi_f)) <= 1e-13 * (1 + np.abs(pc).sum())


def _kind(lev, dof):
    nd = 2 * lev.dim
    node, slot = dof // nd, dof % nd
    c = lev.node_class[node]
    if c == FLUID:
        return "A" if slot < lev.dim else "M"
    return "M" if slot < lev.dim else "K"


def test_restriction_is_transpose_with_interface_rule():
    coarse, fine = build_level(CHANNEL_2D, 0), build_level(CHANNEL_2D, 1)
    P0 = solver.prolongation(coarse, fine).tocsr()
    Pm, R = solver.transfer_operators(coarse, fine)
    nd, dim = 4, 2
    nnc, nnf = coarse.n_nodes * nd, fine.n_nodes * nd
    Rd = R.tocsr()
    # pressure part and masked P: exact transposes of the injection
    assert abs(Rd[nnc:, nnf:] - P0[nnf:, nnc:].T).max() == 0
    keep = sp.diags((~fine.dir_mask).astype(float)) @ P0 @ sp.diags((~coarse.dir_mask).astype(float))
    assert abs(Pm - keep).max() == 0
    # node part: R[(C,sc),(f,sf)] = phi_C(f) iff same component and same equation kind
    S = solver.scalar_node_prolongation(coarse, fine).tocsr()
    cross = 0
    for C in range(coarse.n_nodes):
        for sc in range(nd):
            row = C * nd + sc
            a, b = Rd.indptr[row], Rd.indptr[row + 1]
            got = dict(zip(Rd.indices[a:b], Rd.data[a:b]))
            want = {}
            if not coarse.dir_mask[row]:
                col = S[:, C].tocoo()
                for f, w in zip(col.row, col.data):
                    for sf in range(nd):
                        if sf % dim != sc % dim or fine.dir_mask[f * nd + sf]:
                            continue
                        if _kind(coarse, row) == _kind(fine, f * nd + sf):
                            want[f * nd + sf] = w
                            if sf != sc:
                                cross += 1
            assert got.keys() == want.keys()
            for k in got:
                assert got[k] == want[k]
    assert cross > 0   # interface momentum rows gather fine fluid u-rows


@pytest.mark.parametrize("prob", [CHANNEL_2D, replace(SMALL_3D, levels=2)], ids=["2d", "3d"])
def test_galerkin_equals_rediscretisation_at_zero(prob):
    coarse, fine = build_level(prob, 0), build_level(prob, 1)
    Pm, R = solver.transfer_operators(coarse, fine)
    _, Jf = fem.assemble(prob, fine, np.zeros(fine.N))
    Jg = solver.galerkin(Jf, Pm, R, coarse).toarray()
    _, Jc = fem.assemble(prob, coarse, np.zeros(coarse.N))
    Jc = Jc.toarray()
    nd = 2 * prob.dim
    free = ~coarse.dir_mask
    scale = np.ones(coarse.N)
    for C in range(coarse.n_nodes):
        if coarse.node_class[C] == FLUID:
            scale[C * nd: C * nd + prob.dim] = 2.0 ** prob.dim     # ALE rows: k_fine = 2^dim k_coarse
    A = Jg[np.ix_(free, free)]
    B = (scale[:, None] * Jc)[np.ix_(free, free)]
    assert np.abs(A - B).max() <= 1e-9 * np.abs(B).max()
    # coarse Dirichlet rows are identity rows, their columns empty
    d = np.nonzero(coarse.dir_mask)[0]
    assert np.all(Jg[d][:, d] == np.eye(len(d)))
    assert np.all(Jg[np.ix_(free, d)] == 0)


def _small_system():
    prob = replace(CHANNEL_2D, levels=1)
    lev = build_level(prob, 0)
    y = initial_state(prob, lev, noise(lev.N, 0))
    r, J = fem.assemble(prob, lev, y)
    return lev, J.tocsr(), -r


def test_ras_one_subdomain_one_step():
    lev, J, b = _small_system()
    ops = solver.LevelOps(lev=lev, J=J, patches=[Patch(elems=np.arange(lev.n_elem), dofs=np.arange(lev.N),
                                                     owned=np.ones(lev.N, dtype=bool), solid=False)])
    solver.factor_patches(ops)
    x = np.zeros(lev.N)
    x = x + 1.0 * solver.ras_apply(ops, b - J @ x)
    assert np.linalg.norm(b - J @ x) <= 1e-12 * np.linalg.norm(b)


def test_ras_matches_dense_formula():
    lev, J, b = _small_system()
    from oracle.mesh import build_patches
    pts = build_patches(lev, (8, 4))
    assert len(pts) >= 2
    ops = solver.LevelOps(lev=lev, J=J, patches=pts)
    solver.factor_patches(ops)
    Jd = J.toarray()
    M = np.zeros_like(Jd)
    for pt in pts:
        Rd = np.zeros((len(pt.dofs), lev.N))
        Rd[np.arange(len(pt.dofs)), pt.dofs] = 1.0
        R0 = Rd * pt.owned[:, None]
        M += R0.T @ np.linalg.inv(Rd @ Jd @ Rd.T) @ Rd
    r = np.random.default_rng(1).standard_normal(lev.N)
    want = M @ r
    got = solver.ras_apply(ops, r)
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)


def test_fgmres_identity_diagonal():
    A = sp.diags([1.0, 2.0, 3.0, 4.0, 5.0]).tocsr()
    b = np.ones(5)
    x, st = solver.fgmres(A, b, lambda v: v, restart=30, rtol=1e-12)
    assert st.iters <= 5
    assert np.allclose(x, 1.0 / np.arange(1, 6), rtol=1e-12)


def test_fgmres_vcycle_matches_direct_solve():
    prob, opts = CONFIGS["channel2d_l3"]
    prob = replace(prob, levels=2)
    orc = solver.Oracle(prob, opts)
    y = initial_state(prob, orc.fine, noise(orc.fine.N, 0))
    r, J = orc.assemble(y)
    orc.factor()
    x, st = orc.solve(-r, rtol=1e-12)
    xs = solver.direct_solve(J, -r)
    assert st.rel_res <= 1e-12
    assert st.iters < 30
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_newton_converges_quadratically():
    prob, opts = CONFIGS["channel2d_l3"]
    prob = replace(prob, levels=2)
    orc = solver.Oracle(prob, opts)
    lev = orc.fine
    y0 = np.zeros(lev.N)
    y0[lev.dir_mask] = lev.dir_val[lev.dir_mask]
    y, hist = orc.newton(y0, tol=1e-8, linear="direct")
    rels = [h[0] for h in hist]
    assert rels[-1] < 1e-8 and len(rels) <= 15
    # quadratic tail of the exact Newton method (exact Jacobian): the last
    # steps square the relative update up to a modest factor
    assert rels[-1] < 1e3 * rels[-2] ** 2
    assert rels[-2] < rels[-3] * 1e-1


# ----------------------------------------------------------------------------
# left-preconditioned GMRES(m) (Sec. 4.1)
# ----------------------------------------------------------------------------

def _krylov_min(A, P, b, x0, k):
    """Brute force: x in x0 + K_k(P A, P r0) minimising ||P (b - A x)||, from
    an orthonormal basis of the explicit Krylov vectors (numpy QR + lstsq)."""
    r = P @ (b - A @ x0)
    K = [r]
    for _ in range(k - 1):
        K.append(P @ (A @ K[-1]))
    Q, _ = np.linalg.qr(np.array(K).T)
    y, *_ = np.linalg.lstsq(P @ A @ Q, r, rcond=None)
    return x0 + Q @ y


@pytest.mark.parametrize("passes", [1, 2])
def test_gmres_left_minimises_the_preconditioned_residual(passes):
    """After k steps without restart the iterate minimises the left-
    preconditioned residual over the Krylov space; with restart m the same
    holds cycle by cycle, each cycle starting from the previous iterate."""
    from oracle.solver import gmres_left
    rng = np.random.default_rng(1)
    n = 30
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.5
    P = np.linalg.inv(np.eye(n) * 3 + np.triu(rng.standard_normal((n, n)) * 0.3))
    b = rng.standard_normal(n)
    x, st = gmres_left(A, b, lambda v: P @ v, restart=20, rtol=1e-30, max_iters=7, gs_passes=passes)
    assert st.iters == 7
    want = _krylov_min(A, P, b, np.zeros(n), 7)
    assert np.linalg.norm(x - want) <= 1e-10 * np.linalg.norm(want)
    x, st = gmres_left(A, b, lambda v: P @ v, restart=3, rtol=1e-30, max_iters=6, gs_passes=passes)
    x1 = _krylov_min(A, P, b, np.zeros(n), 3)
    want = _krylov_min(A, P, b, x1, 3)
    assert np.linalg.norm(x - want) <= 1e-10 * np.linalg.norm(want)


def test_gmres_left_stopping_rule():
    """It stops at the first step whose minimal left-preconditioned residual
    is below rtol times the initial one (brute force over k), and reports
    that ratio; identity preconditioning of a 5 x 5 diagonal system takes at
    most 5 steps."""
    from oracle.solver import gmres_left
    rng = np.random.default_rng(2)
    n = 25
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.4
    P = np.diag(1.0 / np.diag(A))
    b = rng.standard_normal(n)
    x, st = gmres_left(A, b, lambda v: P @ v, restart=50, rtol=1e-6, max_iters=50)
    r0 = np.linalg.norm(P @ b)
    ks = [k for k in range(1, n + 1)
          if np.linalg.norm(P @ (b - A @ _krylov_min(A, P, b, np.zeros(n), k))) < 1e-6 * r0]
    assert st.iters == ks[0]
    assert st.rel_res == pytest.approx(np.linalg.norm(P @ (b - A @ x)) / r0, rel=1e-8)
    D = np.diag([1.0, 2.0, 3.0, 4.0, 5.0])
    _, st = gmres_left(D, np.ones(5), lambda v: v, restart=10, rtol=1e-12)
    assert st.iters <= 5 and st.rel_res < 1e-12


# ----------------------------------------------------------------------------
# nested iteration (full multigrid) for the steady problem (Sec. 3)
# ----------------------------------------------------------------------------

def test_state_injection_keeps_boundary_data_and_coarse_fields():
    """Injecting a coarse state whose node values are a global biquadratic
    field (in every level's Q2 space) reproduces that field at every free
    fine unknown - including the fine nodes next to the boundary, whose
    coarse stencil holds boundary nodes, so boundary values are carried, not
    dropped as in the correction prolongation - and sets every fine
    Dirichlet unknown to its data."""
    from oracle.mesh import build_level
    from oracle.solver import inject_state, transfer_operators
    from paper_1709_05660_gb300.workloads import Problem
    prob = Problem(levels=2, U=0.3)
    c, f = build_level(prob, 0), build_level(prob, 1)
    nd = 4
    q = lambda xy, s_: (0.3 + 0.7 * xy[:, 0] - 1.1 * xy[:, 1] ** 2 + 0.2 * xy[:, 0] * xy[:, 1]
                        + 0.05 * xy[:, 0] ** 2 * xy[:, 1] ** 2) * (s_ + 1)
    yc = np.zeros(c.N)
    for s_ in range(nd):
        yc[s_:c.n_nodes * nd:nd] = q(c.node_xyz, s_)
    yf = inject_state(c, f, yc)
    assert np.array_equal(yf[f.dir_mask], f.dir_val[f.dir_mask])
    want = np.zeros(f.N)
    for s_ in range(nd):
        want[s_:f.n_nodes * nd:nd] = q(f.node_xyz, s_)
    free = ~f.dir_mask
    free[f.n_nodes * nd:] = False
    assert np.max(np.abs(yf[free] - want[free])) <= 1e-13 * np.max(np.abs(want))
    # the masked correction prolongation differs exactly where coarse boundary
    # values enter free fine unknowns
    P, _ = transfer_operators(c, f)
    assert np.max(np.abs((P @ yc)[free] - want[free])) > 1e-3


def test_fmg_reaches_the_steady_state_of_plain_newton():
    """Nested iteration from the coarsest mesh ends at the same discrete
    steady state as plain Newton on the finest mesh from the lift, with no
    more finest-level Newton steps."""
    from oracle.mesh import initial_state
    from oracle.solver import Oracle, fmg_newton
    from paper_1709_05660_gb300.workloads import Problem, SolverOpts
    prob, opts = Problem(levels=3, mu_s=5e5, U=0.2), SolverOpts(tile=(2, 2))
    y_fmg, hists = fmg_newton(prob, opts, tol=1e-10)
    assert len(hists) == 3 and all(h[-1][0] < 1e-10 for h in hists)
    orc = Oracle(prob, opts)
    y_pl, hist_pl = orc.newton(initial_state(prob, orc.fine, np.zeros(orc.fine.N)), tol=1e-10, linear="direct")
    assert np.linalg.norm(y_fmg - y_pl) <= 1e-9 * np.linalg.norm(y_pl)
    assert len(hists[-1]) <= len(hist_pl)
    r, _ = orc.assemble(y_fmg)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(orc.assemble(initial_state(prob, orc.fine, np.zeros(orc.fine.N)))[0])


# ----------------------------------------------------------------------------
# ILU(0) local solver of the fluid blocks (Sec. 3.3, 4.1)
# ----------------------------------------------------------------------------

def test_ilu0_defining_property_on_a_block_pattern():
    """On a random block-sparse pattern (with the diagonal): L is unit lower
    and U upper triangular, both zero outside the pattern, and L U equals B at
    every pattern entry (the entries outside hold the dropped fill)."""
    from oracle.solver import ilu0
    rng = np.random.default_rng(5)
    nb, b = 12, 4
    bm = rng.uniform(size=(nb, nb)) < 0.35
    bm |= bm.T
    np.fill_diagonal(bm, True)
    mask = np.kron(bm, np.ones((b, b), dtype=bool))
    n = nb * b
    B = rng.standard_normal((n, n)) * mask + np.eye(n) * 8.0
    L, U = ilu0(B, mask)
    assert np.allclose(np.triu(L, 1), 0.0) and np.allclose(np.diag(L), 1.0)
    assert np.allclose(np.tril(U, -1), 0.0)
    assert np.all(L[~mask] == 0.0) and np.all(U[~mask] == 0.0)
    LU = L @ U
    assert np.max(np.abs(LU[mask] - B[mask])) <= 1e-12 * np.max(np.abs(B))
    assert np.max(np.abs(LU[~mask])) > 1e-6          # fill was dropped somewhere


def test_ilu0_special_cases():
    """A full pattern gives the LU factorisation without pivoting (diagonally
    dominant, so partial pivoting keeps the diagonal: scipy's LU with P = I);
    a tridiagonal pattern has no fill, so ILU(0) solves exactly."""
    from oracle.solver import ilu0
    rng = np.random.default_rng(6)
    n = 20
    B = rng.standard_normal((n, n)) + np.eye(n) * 3 * n
    L, U = ilu0(B, np.ones((n, n), dtype=bool))
    P, L2, U2 = sla.lu(B)
    assert np.array_equal(P, np.eye(n))
    assert np.allclose(L, L2, atol=1e-13) and np.allclose(U, U2, rtol=1e-12, atol=1e-12)
    T = np.diag(rng.uniform(2, 3, n)) + np.diag(rng.standard_normal(n - 1), 1) + np.diag(rng.standard_normal(n - 1), -1)
    mask = T != 0.0
    L, U = ilu0(T, mask)
    rhs = rng.standard_normal(n)
    x = sla.solve_triangular(U, sla.solve_triangular(L, rhs, lower=True, unit_diagonal=True))
    band = np.zeros((3, n))
    band[0, 1:] = np.diag(T, 1)
    band[1] = np.diag(T)
    band[2, :-1] = np.diag(T, -1)
    assert np.allclose(x, sla.solve_banded((1, 1), band, rhs), rtol=1e-12)


def test_fluid_ilu_vcycle_solves_with_fgmres():
    """With ILU(0) fluid blocks (LU for solid ones) the V-cycle is still a
    preconditioner under which FGMRES reaches the direct solution; the solid
    blocks keep their exact LU."""
    from dataclasses import replace as _r
    from oracle.mesh import initial_state
    from oracle.solver import Oracle, direct_solve
    from paper_1709_05660_gb300.workloads import CONFIGS, noise
    prob, opts = CONFIGS["channel2d_l3"]
    orc = Oracle(_r(prob, levels=2), _r(opts, local_solver=1))
    y0 = initial_state(orc.prob, orc.fine, noise(orc.fine.N, 0))
    r, J = orc.assemble(y0)
    orc.factor()
    kinds = [isinstance(lu, tuple) and isinstance(lu[0], str) for lu in orc.ops[1].lu]
    solid = [pt.solid for pt in orc.ops[1].patches]
    assert kinds == [not s for s in solid] and any(solid) and not all(solid)
    x, st = orc.solve(-r)
    xs = direct_solve(J, -r)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
