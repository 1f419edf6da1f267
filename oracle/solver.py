"""Oracle: multigrid transfers, Galerkin coarse operators, Richardson-Schwarz
smoother, V-cycle, FGMRES, direct solve and Newton driver.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Prolongation (Sec. 3.2): the natural injection of the coarse Q2 / P1disc
  spaces into the fine ones: P_ij = coarse basis j evaluated at fine node i
  (per field component); a P1disc child inherits its parent's linear
  function.  Entries touching a Dirichlet unknown (fine row or coarse
  column) are dropped.
* Restriction (Sec. 3.2): the transpose of the prolongation with the
  interface rule of the block structure in Sec. 3.2: a coarse equation only
  gathers fine equations of the same kind.  In the shuffled row layout used
  here (see ``fem``) that means: momentum rows gather momentum rows (for a
  coarse interface / solid node they sit in d-rows, for a fluid node in
  u-rows); the coarse solid kinematic rows (u-rows of solid / interface
  nodes) gather only fine kinematic rows, never the fine fluid ALE rows;
  ALE rows gather ALE rows.  Dirichlet rows are dropped.
* Galerkin coarse operator J_{l-1} = R J_l P (Sec. 3.2), plus identity rows
  at coarse Dirichlet unknowns.
* Restricted additive Schwarz preconditioned Richardson (Sec. 3.3):
  x <- x + omega sum_k (R^0_k)^T B_k^{-1} R^delta_k (b - J x), with B_k the
  dense restriction of J to R^delta_k solved by partial-pivot LU.
* V-cycle: nu_pre smoothing steps from x = 0, residual, restriction,
  recursion, prolongation, nu_post smoothing steps; direct solve on level 0
  (Sec. 3, 4.1).
* FGMRES(m), right preconditioned, classical Gram-Schmidt applied twice,
  zero initial guess, true residual checked at every restart / exit.
  (The paper uses left-preconditioned GMRES with one classical Gram-Schmidt
  pass, Sec. 4.1; the flexible right-preconditioned form with a second pass
  is this build's reading, needed for relative tolerances near 1e-10.)
* Left-preconditioned GMRES(m) with classical Gram-Schmidt and the test on
  the left-preconditioned residual: the paper's own Krylov setting (Sec.
  4.1), used for its parameter studies (Sec. 4.4).
* Direct solve x* = J^{-1} b: sparse LU (SuperLU) plus two steps of
  iterative refinement - the plain definition the iterative solve approaches.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem
from .fem import q2_1d
from .mesh import FLUID, IFACE, SOLID, Level, Patch, build_hierarchy, build_patches


# ----------------------------------------------------------------------------
# transfers
# ----------------------------------------------------------------------------

def scalar_node_prolongation(coarse: Level, fine: Level) -> sp.csr_matrix:
    """(fine nodes x coarse nodes) matrix of coarse Q2 basis values at fine
    nodes.  Along each axis the fine Q2 nodes sit at the quarter points of
    the coarse cell (reference coordinates -1, -1/2, 0, 1/2, 1)."""
    dim = fine.dim
    axes = []
    for d in range(dim):
        nf = fine.nodes_ax[d]
        nc_cells = coarse.cells[d]
        rows, cols, vals = [], [], []
        for i in range(nf):
            ec = min(i // 4, nc_cells - 1)
            xi = -1.0 + (i - 4 * ec) / 2.0
            L = q2_1d(xi)
            for m in range(3):
                if L[m] != 0.0:
                    rows.append(i)
                    cols.append(2 * ec + m)
                    vals.append(L[m])
        axes.append(sp.csr_matrix((vals, (rows, cols)), shape=(nf, coarse.nodes_ax[d])))
    # lexicographic x fastest: node = i + nx * (j + ny * k) -> kron(z, y, x)
    M = axes[0]
    for d in range(1, dim):
        M = sp.kron(axes[d], M, format="csr")
    M.eliminate_zeros()
    return M.tocsr()


def pressure_prolongation(coarse: Level, fine: Level) -> sp.csr_matrix:
    """P1disc: child coefficients (1, xi, eta..) from parent coefficients.
    Child with position s_d in {0,1} along axis d: xi_c = (xi_f + (2 s_d - 1)) / 2."""
    dim = fine.dim
    rows, cols, vals = [], [], []
    for ef in range(fine.n_elem):
        r = ef
        fi = []
        for c in fine.cells:
            fi.append(r % c)
            r //= c
        ci = [f // 2 for f in fi]
        s = [f % 2 for f in fi]
        ec = 0
        stride = 1
        for d in range(dim):
            ec += ci[d] * stride
            stride *= coarse.cells[d]
        fb = fine.n_nodes * 2 * dim + ef * (dim + 1)
        cb = coarse.n_nodes * 2 * dim + ec * (dim + 1)
        # constant term
        rows.append(fb); cols.append(cb); vals.append(1.0)
        for d in range(dim):
            sig = 2 * s[d] - 1
            rows.append(fb); cols.append(cb + 1 + d); vals.append(0.5 * sig)
            rows.append(fb + 1 + d); cols.append(cb + 1 + d); vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.N, coarse.N))


def prolongation(coarse: Level, fine: Level) -> sp.csr_matrix:
    """Full (unmasked) natural injection on all unknowns."""
    nd = 2 * fine.dim
    S = scalar_node_prolongation(coarse, fine).tocoo()
    rows = np.concatenate([S.row * nd + c for c in range(nd)])
    cols = np.concatenate([S.col * nd + c for c in range(nd)])
    vals = np.concatenate([S.data for _ in range(nd)])
    Pn = sp.csr_matrix((vals, (rows, cols)), shape=(fine.N, coarse.N))
    return (Pn + pressure_prolongation(coarse, fine)).tocsr()


def _row_kind(lev: Level, dofs: np.ndarray) -> np.ndarray:
    """Equation kind held by each node row: 0 momentum, 1 solid kinematic,
    2 ALE (shuffled layout)."""
    nd = 2 * lev.dim
    node = dofs // nd
    slot = dofs % nd
    cls = lev.node_class[node]
    is_d = slot < lev.dim
    kind = np.where(cls == FLUID, np.where(is_d, 2, 0), np.where(is_d, 0, 1))
    return kind


def transfer_operators(coarse: Level, fine: Level):
    """Masked prolongation P (fine x coarse) and interface-aware restriction
    R (coarse x fine)."""
    P = prolongation(coarse, fine).tocoo()
    keep = ~fine.dir_mask[P.row] & ~coarse.dir_mask[P.col]
    Pm = sp.csr_matrix((P.data[keep], (P.row[keep], P.col[keep])), shape=P.shape)

    # R: start from the unmasked injection transposed, node part rebuilt with
    # the equation-kind rule (same component, same kind).
    nd = 2 * fine.dim
    dim = fine.dim
    S = scalar_node_prolongation(coarse, fine).tocoo()   # (fine node f, coarse node C)
    rows, cols, vals = [], [], []
    for sc in range(nd):                       # coarse slot
        comp = sc % dim
        for sf in (comp, dim + comp):          # fine slots of the same component
            cr = S.col * nd + sc
            fr = S.row * nd + sf
            kc = _row_kind(coarse, cr)
            kf = _row_kind(fine, fr)
            ok = (kc == kf) & ~coarse.dir_mask[cr] & ~fine.dir_mask[fr]
            rows.append(cr[ok]); cols.append(fr[ok]); vals.append(S.data[ok])
    Pp = pressure_prolongation(coarse, fine).tocoo()
    rows.append(Pp.col); cols.append(Pp.row); vals.append(Pp.data)
    R = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(coarse.N, fine.N))
    return Pm, R


def galerkin(Jf: sp.csr_matrix, P: sp.csr_matrix, R: sp.csr_matrix, coarse: Level) -> sp.csr_matrix:
    """J_{l-1} = R J_l P (Sec. 3.2) on the coarse FE pattern, identity rows at
    coarse Dirichlet unknowns."""
    Jc = (R @ Jf @ P).tocoo()
    J = fem.place_on_pattern(fem.fe_pattern(coarse), Jc)
    fem.apply_dirichlet_rows(J, coarse.dir_mask)
    return J


# ----------------------------------------------------------------------------
# smoother, V-cycle, FGMRES
# ----------------------------------------------------------------------------

@dataclass
class LevelOps:
    lev: Level
    J: sp.csr_matrix
    patches: List[Patch] = field(default_factory=list)
    lu: list = field(default_factory=list)     # per patch (lu, piv)
    P: Optional[sp.csr_matrix] = None           # to this level from level-1
    R: Optional[sp.csr_matrix] = None
    coarse_lu: object = None


def ilu0(B: np.ndarray, mask: np.ndarray):
    """Incomplete LU factorisation with zero fill (Sec. 3.3, 4.1: the
    approximate local solver of the fluid subdomains): Gaussian elimination
    without pivoting in which every entry outside the sparsity pattern
    `mask` (which must hold the diagonal) stays zero.  Row by row (i), each
    earlier row k of the pattern first scales the entry (i, k) by 1 / u_kk,
    then subtracts l_ik u_kj from the pattern entries (i, j), j > k.
    Returns (L, U): L unit lower triangular, U upper triangular, both
    supported on the pattern, with (L U)_ij = B_ij on the pattern."""
    A = np.array(B, dtype=np.float64)
    n = A.shape[0]
    assert np.all(np.diag(mask))
    A[~mask] = 0.0
    for i in range(1, n):
        for k in np.nonzero(mask[i, :i])[0]:
            A[i, k] /= A[k, k]
            A[i, k + 1:] -= A[i, k] * A[k, k + 1:] * mask[i, k + 1:]
    L = np.tril(A, -1) + np.eye(n)
    U = np.triu(A)
    return L, U


def patch_pattern(ops: LevelOps, pt) -> np.ndarray:
    """Sparsity pattern of a Schwarz block: the FE pattern of the level
    (Sec. 3.1 blocks) restricted to R^delta_k, with the diagonal added (the
    element pressure rows have no pressure-pressure entries)."""
    P = fem.fe_pattern(ops.lev)
    Pk = P[pt.dofs][:, pt.dofs]
    mask = np.zeros((len(pt.dofs), len(pt.dofs)), dtype=bool)
    coo = Pk.tocoo()
    mask[coo.row, coo.col] = True
    np.fill_diagonal(mask, True)
    return mask


def factor_patches(ops: LevelOps, fluid_ilu: bool = False) -> None:
    """Local solvers of the Schwarz blocks: partial-pivot LU of every block,
    or (fluid_ilu) ILU(0) of the fluid blocks and LU of the solid ones, the
    setting of Sec. 3.3 and 4.1."""
    Jd = ops.J.tocsr()
    ops.lu = []
    for pt in ops.patches:
        B = Jd[pt.dofs][:, pt.dofs].toarray()
        if fluid_ilu and not pt.solid:
            ops.lu.append(("ilu",) + ilu0(B, patch_pattern(ops, pt)))
        else:
            ops.lu.append(sla.lu_factor(B, check_finite=True))


def ras_apply(ops: LevelOps, r: np.ndarray) -> np.ndarray:
    """sum_k (R^0_k)^T B_k^{-1} R^delta_k r  (restricted additive Schwarz);
    an ILU(0) block applies U^{-1} L^{-1} in place of B_k^{-1}."""
    out = np.zeros_like(r)
    for pt, lu in zip(ops.patches, ops.lu):
        if isinstance(lu, tuple) and lu and isinstance(lu[0], str):
            _, L, U = lu
            z = sla.solve_triangular(U, sla.solve_triangular(L, r[pt.dofs], lower=True, unit_diagonal=True))
        else:
            z = sla.lu_solve(lu, r[pt.dofs])
        out[pt.dofs[pt.owned]] += z[pt.owned]
    return out


def vcycle(levels: List[LevelOps], l: int, b: np.ndarray, opts) -> np.ndarray:
    ops = levels[l]
    if l == 0:
        return sla.lu_solve(ops.coarse_lu, b)
    x = np.zeros_like(b)
    for s in range(opts.n_pre):
        r = b if s == 0 else b - ops.J @ x
        x = x + opts.omega * ras_apply(ops, r)
    r = b - ops.J @ x
    xc = vcycle(levels, l - 1, ops.R @ r, opts)
    x = x + ops.P @ xc
    for s in range(opts.n_post):
        r = b - ops.J @ x
        x = x + opts.omega * ras_apply(ops, r)
    return x


@dataclass
class SolveStats:
    iters: int = 0
    restarts: int = 0
    rel_res: float = np.nan
    history: list = field(default_factory=list)
    true_rel_res: float = np.nan


def fgmres(A, b: np.ndarray, precond, restart: int = 30, rtol: float = 1e-10,
           max_iters: int = 1000, x0: Optional[np.ndarray] = None):
    """Right-preconditioned flexible GMRES with CGS2 (see module doc)."""
    n = len(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    st = SolveStats()
    if bnorm == 0.0:
        st.rel_res = 0.0
        return x, st
    r = b - A @ x
    beta = np.linalg.norm(r)
    st.history.append(beta / bnorm)
    while True:
        if beta <= rtol * bnorm or st.iters >= max_iters:
            st.rel_res = beta / bnorm
            return x, st
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = precond(V[j])
            w = A @ Z[j]
            wnorm0 = np.linalg.norm(w)
            h = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1] @ w
            w = w - V[: j + 1].T @ h2
            h = h + h2
            H[: j + 1, j] = h
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            breakdown = hn <= 1e-14 * wnorm0
            if not breakdown:
                V[j + 1] = w / hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            st.iters += 1
            k = j + 1
            st.history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or breakdown or st.iters >= max_iters:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + Z[:k].T @ y
        r = b - A @ x
        beta = np.linalg.norm(r)
        st.restarts += 1
        if beta <= rtol * bnorm or st.iters >= max_iters:
            st.rel_res = beta / bnorm
            return x, st


def gmres_left(A, b: np.ndarray, precond, restart: int = 10, rtol: float = 1e-4, max_iters: int = 1000,
               gs_passes: int = 1, x0: Optional[np.ndarray] = None):
    """Left-preconditioned restarted GMRES(m), the paper's setting (Sec. 4.1):
    Arnoldi on P^{-1} A with classical Gram-Schmidt (one pass, or two with
    gs_passes = 2), the solution update x += V y, and convergence at step j
    when the left-preconditioned residual r_L^j = P^{-1}(b - A x_j) satisfies
    ||r_L^j|| < rtol ||r_L^0|| (its Givens estimate inside a cycle, the
    recomputed value at each restart).  ``precond(v)`` applies P^{-1}.
    Returns x and SolveStats with rel_res = ||r_L|| / ||r_L^0|` and the true
    relative residual in ``true_rel_res``."""
    n = len(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    st = SolveStats()
    r = precond(b - A @ x)
    r0 = np.linalg.norm(r)
    beta = r0
    st.history.append(1.0)
    if r0 == 0.0:
        st.rel_res = 0.0
        st.true_rel_res = np.linalg.norm(b - A @ x) / max(np.linalg.norm(b), 1e-300)
        return x, st
    while True:
        if beta < rtol * r0 or st.iters >= max_iters:
            break
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            w = precond(A @ V[j])
            wnorm0 = np.linalg.norm(w)
            h = np.zeros(j + 1)
            for _ in range(gs_passes):
                hp = V[: j + 1] @ w
                w = w - V[: j + 1].T @ hp
                h = h + hp
            H[: j + 1, j] = h
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            breakdown = hn <= 1e-14 * wnorm0
            if not breakdown:
                V[j + 1] = w / hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            st.iters += 1
            k = j + 1
            st.history.append(abs(g[j + 1]) / r0)
            if abs(g[j + 1]) < rtol * r0 or breakdown or st.iters >= max_iters:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + V[:k].T @ y
        r = precond(b - A @ x)
        beta = np.linalg.norm(r)
        st.restarts += 1
    st.rel_res = beta / r0
    st.true_rel_res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    return x, st


def direct_solve(A: sp.csr_matrix, b: np.ndarray, refine: int = 2) -> np.ndarray:
    """x* = A^{-1} b by sparse LU plus iterative refinement."""
    lu = spla.splu(A.tocsc())
    x = lu.solve(b)
    for _ in range(refine):
        x = x + lu.solve(b - A @ x)
    return x


# ----------------------------------------------------------------------------
# nested iteration (full multigrid) for the steady nonlinear problem
# ----------------------------------------------------------------------------

def inject_state(coarse: Level, fine: Level, yc: np.ndarray) -> np.ndarray:
    """A coarse state carried to the next finer mesh by the natural injection
    of the nested spaces (Sec. 3.2) - every coarse unknown, boundary values
    included - with the fine Dirichlet unknowns then set to their data."""
    yf = prolongation(coarse, fine) @ yc
    yf[fine.dir_mask] = fine.dir_val[fine.dir_mask]
    return yf


def fmg_newton(prob, opts, tol: float = 1e-8, max_steps: int = 20, linear: str = "direct"):
    """Nested iteration (Sec. 3: full multigrid in the steady case): Newton
    to ||dy|| < tol ||y|| on the coarsest mesh from the boundary-condition
    lift (d = 0, p = 0, u = inflow profile at fluid nodes and the Dirichlet
    data), then on every finer mesh from the injected solution of the
    coarser one.  Mesh level l is solved with the multigrid hierarchy of
    levels 0..l.  Returns the finest state and, per level, the Newton history
    [(||dy|| / ||y||, Krylov iterations), ...]."""
    from dataclasses import replace as _replace
    from .mesh import initial_state
    y, hists, prev = None, [], None
    for l in range(prob.levels):
        orc = Oracle(_replace(prob, levels=l + 1), opts)
        lev = orc.fine
        y0 = initial_state(prob, lev, np.zeros(lev.N)) if prev is None else inject_state(prev, lev, y)
        y, hist = orc.newton(y0, tol=tol, max_steps=max_steps, linear=linear)
        hists.append(hist)
        prev = lev
    return y, hists


# ----------------------------------------------------------------------------
# whole hierarchy
# ----------------------------------------------------------------------------

class Oracle:
    """Hierarchy + operators for one problem (the CPU counterpart of an
    ``fsi_ctx``)."""

    def __init__(self, prob, opts):
        self.prob = prob
        self.opts = opts
        self.levels_mesh = build_hierarchy(prob)
        self.ops: List[LevelOps] = []
        self._transfers = []
        for l in range(1, prob.levels):
            self._transfers.append(transfer_operators(self.levels_mesh[l - 1], self.levels_mesh[l]))
        self._patches = [None] + [build_patches(self.levels_mesh[l], opts.tile)
                                  for l in range(1, prob.levels)]

    @property
    def fine(self) -> Level:
        return self.levels_mesh[-1]

    def assemble(self, y: np.ndarray, source=None, tr=None):
        """Finest r, J and all Galerkin levels (tr: transient history, see
        fem.assemble)."""
        r, J = fem.assemble(self.prob, self.fine, y, source, tr=tr)
        L = self.prob.levels
        Js = [None] * L
        Js[L - 1] = J
        for l in range(L - 1, 0, -1):
            P, R = self._transfers[l - 1]
            Js[l - 1] = galerkin(Js[l], P, R, self.levels_mesh[l - 1])
        self.ops = []
        for l in range(L):
            op = LevelOps(lev=self.levels_mesh[l], J=Js[l])
            if l > 0:
                op.P, op.R = self._transfers[l - 1]
                op.patches = self._patches[l]
            self.ops.append(op)
        return r, J

    def factor(self):
        fluid_ilu = getattr(self.opts, "local_solver", 0) == 1
        for l, op in enumerate(self.ops):
            if l == 0:
                op.coarse_lu = sla.lu_factor(op.J.toarray())
            else:
                factor_patches(op, fluid_ilu)

    def precond(self, v: np.ndarray) -> np.ndarray:
        return vcycle(self.ops, len(self.ops) - 1, v, self.opts)

    def solve(self, b: np.ndarray, rtol: Optional[float] = None):
        """The workload's Krylov method: FGMRES (right preconditioned, CGS2,
        true-residual test) or, with opts.krylov == 1, the paper's
        left-preconditioned GMRES(m) with opts.gs_passes Gram-Schmidt passes."""
        o = self.opts
        rt = o.rtol if rtol is None else rtol
        if getattr(o, "krylov", 0) == 1:
            return gmres_left(self.ops[-1].J, b, self.precond, o.restart, rt, o.max_iters,
                              gs_passes=getattr(o, "gs_passes", 1) or 1)
        return fgmres(self.ops[-1].J, b, self.precond, o.restart, rt, o.max_iters)

    def newton(self, y0: np.ndarray, tol: float = 1e-8, max_steps: int = 20, linear="fgmres"):
        """Exact Newton (Sec. 3.1, 4.1): J dy = -r, y += dy, stop when
        ||dy|| < tol ||y||."""
        y = y0.copy()
        hist = []
        for k in range(max_steps):
            r, J = self.assemble(y)
            if linear == "fgmres":
                self.factor()
                dy, st = self.solve(-r)
                its = st.iters
            else:
                dy = direct_solve(J, -r)
                its = 0
            y = y + dy
            rel = np.linalg.norm(dy) / np.linalg.norm(y)
            hist.append((rel, its))
            if rel < tol:
                break
        return y, hist
