"""Oracle: residual of the monolithic ALE FSI weak form on Q2-P1disc elements
and its exact Jacobian by forward-mode dual numbers.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What is computed (steady case, Sec. 2.3 with zero time derivatives and zero
body forces; the Jacobian is the exact derivative of the discrete residual,
as the paper obtains it by automatic differentiation, Sec. 3):

Kinematics (Sec. 2.1): F = I + grad_hat d, J = det F, B = F F^T.

Solid element (Lagrangian, Sec. 2.2 / 2.3), incompressible Neo-Hookean
sigma = -p I + 2 C1 B or Mooney-Rivlin sigma = -p I + 2 C1 B - 2 C2 B^{-1}
(Sec. 2.2), with C2 = ``mr_c2`` (0: Neo-Hookean) and C1 = mu_s/2 - C2, so
that mu_s = 2 (C1 + C2) stays the shear modulus of the linearised law:
    momentum  (J sigma F^{-T} : grad_hat phi)
              = (( -p J F^{-T} + 2 C1 J F - 2 C2 J F^{-T} F^{-1} F^{-T} ) : grad_hat phi)
              (B F^{-T} = F and B^{-1} F^{-T} = F^{-T} F^{-1} F^{-T})
    mass      ((J - 1) q)
    kinematic (u . psi)                              (steady: d/dt d = 0)
Fluid element (ALE, integrals on the deformed element x = x_hat + d):
    momentum  J [ rho_f ((grad u) u) . phi + sigma_f : grad phi ],
              sigma_f = -p I + mu_f (grad u + grad u^T), grad = F^{-T}-mapped
    mass      J (div u) q
    ALE       k (grad_hat d + grad_hat d^T) : grad_hat psi,  k = 1 / V_el
              (psi vanishes on the interface, Sec. 2.3; ``ale_op = 1`` gives
              the harmonic variant k grad_hat d : grad_hat psi)

Row placement (the shuffled layout J_shuf of Sec. 3.1, whose blocks are the
ones the Schwarz subdomains of Sec. 3.3 are extracted from):
    solid / interface node:  d-rows = momentum (interface: solid + fluid
                             momentum, the I rows), u-rows = solid kinematic
    fluid node:              d-rows = ALE, u-rows = fluid momentum
    element pressure rows:   mass balance of that element.
Dirichlet unknowns get the row e_i^T and residual y_i - g_i (pattern kept).

Transient form (BDF reading of the time-discretised operators of Sec. 2.5;
the paper's own Crank-Nicolson form is not built): with q_t = (a0 q + a1 q_n +
a2 q_{n-1}) / dt (BDF1: 1, -1, 0; BDF2: 3/2, -2, 1/2) applied to nodal values,
    fluid momentum  J [ rho_f (u_t + (grad u)(u - w)) . phi + sigma_f : grad phi ],  w = d_t
    solid momentum  rho_s J u_t . phi + P : grad_hat phi
    kinematic       (u - d_t) . psi
and the inflow Dirichlet data scaled by alpha(t) = (1 + sin 2 pi t) / 2.

Quadrature: 3 Gauss points per axis (the paper does not state its rule; three
points integrate the Q2 x Q2 products exactly on rectangles).
P1disc basis per element: {1, xi, eta(, zeta)} in reference coordinates.
"""
import itertools
from typing import Callable, Optional, Tuple

import numpy as np
import scipy.sparse as sp

from .mesh import FLUID, IFACE, SOLID, Level

GAUSS_X = np.array([-np.sqrt(3.0 / 5.0), 0.0, np.sqrt(3.0 / 5.0)])
GAUSS_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def q2_1d(xi):
    """Quadratic Lagrange basis on [-1, 1] with nodes -1, 0, 1."""
    return np.array([0.5 * xi * (xi - 1.0), 1.0 - xi * xi, 0.5 * xi * (xi + 1.0)])


def q2_1d_deriv(xi):
    return np.array([xi - 0.5, -2.0 * xi, xi + 0.5])


def q2_basis(dim: int, xi: Tuple[float, ...]):
    """Tensor Q2 basis values (3^dim,) and reference gradients (3^dim, dim);
    local node a = i + 3 j (+ 9 k)."""
    L = [q2_1d(x) for x in xi]
    dL = [q2_1d_deriv(x) for x in xi]
    nloc = 3 ** dim
    N = np.zeros(nloc)
    G = np.zeros((nloc, dim))
    for a in range(nloc):
        idx = [(a // 3 ** d) % 3 for d in range(dim)]
        N[a] = np.prod([L[d][idx[d]] for d in range(dim)])
        for j in range(dim):
            G[a, j] = np.prod([(dL[d] if d == j else L[d])[idx[d]] for d in range(dim)])
    return N, G


class Dual:
    """Forward-mode dual number batched over elements: value v (E,),
    derivative g (E, m)."""
    __slots__ = ("v", "g")

    def __init__(self, v, g):
        self.v = v
        self.g = g

    def __add__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v + o.v, self.g + o.g)
        return Dual(self.v + o, self.g)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.g)

    def __sub__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v - o.v, self.g - o.g)
        return Dual(self.v - o, self.g)

    def __rsub__(self, o):
        return Dual(o - self.v, -self.g)

    def __mul__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v * o.v, self.g * o.v[:, None] + o.g * self.v[:, None])
        o = np.asarray(o)
        return Dual(self.v * o, self.g * (o[:, None] if o.ndim == 1 else o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, Dual):
            inv = 1.0 / o.v
            return Dual(self.v * inv, (self.g - o.g * (self.v * inv)[:, None]) * inv[:, None])
        o = np.asarray(o)
        return Dual(self.v / o, self.g / (o[:, None] if o.ndim == 1 else o))


def _det_inv(F):
    """Determinant and inverse of a small matrix of Duals (adjugate formula)."""
    n = len(F)
    if n == 2:
        J = F[0][0] * F[1][1] - F[0][1] * F[1][0]
        adj = [[F[1][1], -F[0][1]], [-F[1][0], F[0][0]]]
    else:
        c = [[None] * 3 for _ in range(3)]
        for i in range(3):
            for j in range(3):
                i1, i2 = [r for r in range(3) if r != i]
                j1, j2 = [r for r in range(3) if r != j]
                c[i][j] = (F[i1][j1] * F[i2][j2] - F[i1][j2] * F[i2][j1]) * (1.0 if (i + j) % 2 == 0 else -1.0)
        J = F[0][0] * c[0][0] + F[0][1] * c[0][1] + F[0][2] * c[0][2]
        adj = [[c[j][i] for j in range(3)] for i in range(3)]
    inv = [[adj[i][j] / J for j in range(n)] for i in range(n)]
    return J, inv


def element_system(prob, lev: Level, elems: np.ndarray, y: np.ndarray,
                   source: Optional[Callable] = None, tr: Optional[dict] = None):
    """Element residuals (E, ndofe) and exact Jacobians (E, ndofe, ndofe) for a
    batch of elements sharing one material.

    ``source(xhat) -> (f_mom (E, dim), g_mass (E,), g_ale (E, dim) | None)``
    is an optional body force / mass / mesh-equation source used only by
    manufactured-solution tests; it adds -(rho f, phi) to the momentum rows,
    -(g, q) to the mass rows and -(g_ale, psi) to the ALE rows.

    ``tr = dict(yn=..., ynm1=..., a=(a0, a1, a2), dt=...)`` switches on the
    transient (BDF) terms; ``tr = dict(scheme="cn", yn=..., dt=...)`` the
    paper's Crank-Nicolson form (see ``cn_terms``); ``None`` is the steady
    form.
    """
    dim = lev.dim
    n = dim
    nd = 2 * dim
    nloc = 3 ** dim
    m = nd * nloc + dim + 1
    E = len(elems)
    solid = bool(lev.elem_solid[elems[0]])
    assert np.all(lev.elem_solid[elems] == solid)
    h = lev.elem_h[elems]                        # (E, dim)
    lo = lev.elem_lo[elems]
    vol = np.prod(h, axis=1)
    kale = 1.0 / vol
    ye = y[lev.elem_dofs[elems]]                 # (E, m)
    cn = tr is not None and tr.get("scheme") == "cn"
    bdf = tr is not None and not cn
    if bdf:
        a0, a1, a2 = tr["a"]
        idt = 1.0 / tr["dt"]
        yold = (a1 * tr["yn"] + a2 * tr["ynm1"])[lev.elem_dofs[elems]]   # constant part of q_t * dt
    if cn:
        idt = 1.0 / tr["dt"]
        yne = tr["yn"][lev.elem_dofs[elems]]                            # state at t_n (constants)
    iface = lev.node_class[lev.elem_nodes[elems]] == IFACE   # (E, nloc)

    Rv = np.zeros((E, m))
    Rg = np.zeros((E, m, m))
    eye_cols = np.arange(m)

    def field(coef, comp):
        """Dual of sum_a coef[:, a] * y[a*nd + comp]; coef (E, nloc)."""
        cols = np.arange(nloc) * nd + comp
        g = np.zeros((E, m))
        g[:, cols] = coef
        return Dual(np.einsum("ea,ea->e", coef, ye[:, cols]), g)

    def pfield(psi):
        cols = nd * nloc + np.arange(dim + 1)
        g = np.zeros((E, m))
        g[:, cols] = psi[None, :]
        return Dual(ye[:, cols] @ psi, g)

    def cfield(coef, comp):
        """Value of the t_n state: sum_a coef[:, a] * y_n[a*nd + comp]."""
        cols = np.arange(nloc) * nd + comp
        return np.einsum("ea,ea->e", coef, yne[:, cols])

    def add_rows(rows, val: Dual, test):
        """R[rows] += val * test; rows (nloc,) or (E, nloc) with -1 = skip,
        test (E, nloc)."""
        if not isinstance(val, Dual):
            val = Dual(np.asarray(val), np.zeros((E, m)))
        tv = val.v[:, None] * test                            # (E, nloc)
        tg = val.g[:, None, :] * test[:, :, None]             # (E, nloc, m)
        if rows.ndim == 1:
            Rv[:, rows] += tv
            Rg[:, rows, :] += tg
        else:
            ee, aa = np.nonzero(rows >= 0)
            rr = rows[ee, aa]
            np.add.at(Rv, (ee, rr), tv[ee, aa])
            np.add.at(Rg, (ee, rr), tg[ee, aa])

    a_idx = np.arange(nloc)
    for q in itertools.product(range(3), repeat=dim):
        xi = tuple(GAUSS_X[q[d]] for d in range(dim))
        wq = np.prod([GAUSS_W[q[d]] for d in range(dim)]) * vol / 2 ** dim   # (E,)
        Nq, Gref = q2_basis(dim, xi)
        Gh = Gref[None, :, :] * (2.0 / h)[:, None, :]           # (E, nloc, dim)
        Nb = np.broadcast_to(Nq[None, :], (E, nloc))
        psi = np.array((1.0,) + xi)
        gd = [[field(Gh[:, :, j], i) for j in range(n)] for i in range(n)]
        gu = [[field(Gh[:, :, j], n + i) for j in range(n)] for i in range(n)]
        u = [field(Nb, n + i) for i in range(n)]
        if bdf:
            # nodal BDF time derivatives interpolated at the quadrature point
            ut = [(field(Nb, n + i) * a0 + np.einsum("ea,a->e", yold[:, np.arange(nloc) * nd + n + i], Nq)) * idt
                  for i in range(n)]
            dt_ = [(field(Nb, i) * a0 + np.einsum("ea,a->e", yold[:, np.arange(nloc) * nd + i], Nq)) * idt
                   for i in range(n)]
        p = pfield(psi)
        F = [[gd[i][j] + (1.0 if i == j else 0.0) for j in range(n)] for i in range(n)]
        J, Finv = _det_inv(F)
        if cn:
            # the t_n state (constants) and the mesh velocity w = (d - d_n) / dt
            gdn = [[cfield(Gh[:, :, j], i) for j in range(n)] for i in range(n)]
            un = [cfield(Nb, n + i) for i in range(n)]
            pn = yne[:, nd * nloc + np.arange(dim + 1)] @ psi
            Fn = [[gdn[i][j] + (1.0 if i == j else 0.0) for j in range(n)] for i in range(n)]
            Jn, Finvn = _det_inv(Fn)
            w = [(field(Nb, i) - cfield(Nb, i)) * idt for i in range(n)]
            gw = [[(gd[i][j] - gdn[i][j]) * idt for j in range(n)] for i in range(n)]
        if solid:
            T = _solid_piola(prob, F, Finv, J, p, n)
            if cn:
                Tn = _solid_piola(prob, Fn, Finvn, Jn, pn, n)
            for c in range(n):
                for j in range(n):
                    Tc = T[c][j] if not cn else T[c][j] * 0.5 + Tn[c][j] * 0.5
                    add_rows(a_idx * nd + c, Tc * wq, Gh[:, :, j])
                if cn:
                    # (rho J u)_{n+1} - (rho J u)_n over dt; kinematic -w + (u + u_n) / 2
                    add_rows(a_idx * nd + c, (u[c] * J - un[c] * Jn) * (prob.rho_s * idt * wq), Nb)
                    add_rows(a_idx * nd + n + c, ((u[c] + un[c]) * 0.5 - w[c]) * wq, Nb)
                    continue
                kin = u[c] if not bdf else u[c] - dt_[c]
                add_rows(a_idx * nd + n + c, kin * wq, Nb)
                if bdf:
                    add_rows(a_idx * nd + c, ut[c] * J * (prob.rho_s * wq), Nb)
            mass = J - 1.0
        else:
            gux = [[None] * n for _ in range(n)]
            for i in range(n):
                for j in range(n):
                    s = gu[i][0] * Finv[0][j]
                    for k in range(1, n):
                        s = s + gu[i][k] * Finv[k][j]
                    gux[i][j] = s
            div = gux[0][0]
            for i in range(1, n):
                div = div + gux[i][i]
            # sigma_f and J sigma_f F^{-T} (so that sigma : grad phi = (J sigma F^{-T}) : grad_hat phi / J)
            sig = [[gux[i][j] * prob.mu_f + gux[j][i] * prob.mu_f for j in range(n)] for i in range(n)]
            for i in range(n):
                sig[i][i] = sig[i][i] - p
            mom_rows = np.where(iface, a_idx[None, :] * nd, a_idx[None, :] * nd + n)
            ale_rows = np.where(iface, -1, a_idx[None, :] * nd)
            if cn:
                gun = [[cfield(Gh[:, :, j], n + i) for j in range(n)] for i in range(n)]
                guxn = [[sum(gun[i][k] * Finvn[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
                sign = [[prob.mu_f * (guxn[i][j] + guxn[j][i]) - (pn if i == j else 0.0) for j in range(n)]
                        for i in range(n)]
                # div w on the two meshes (grad = grad_hat F^{-1})
                divw1 = gw[0][0] * Finv[0][0]
                divwn = gw[0][0] * Finvn[0][0]
                for i in range(n):
                    for k in range(n):
                        if i == 0 and k == 0:
                            continue
                        divw1 = divw1 + gw[i][k] * Finv[k][i]
                        divwn = divwn + gw[i][k] * Finvn[k][i]
            adv = u if not bdf else [u[j] - dt_[j] for j in range(n)]   # u - w
            for c in range(n):
                rows_c = mom_rows + c
                if cn:
                    # conservative ALE form: (rho J u)_{n+1} - (rho J u)_n over dt,
                    # -(div w) u and [(u - w) . grad] u averaged over t_{n+1}, t_n
                    conv1 = gux[c][0] * (u[0] - w[0])
                    convn = -(w[0] - un[0]) * guxn[c][0]
                    for j in range(1, n):
                        conv1 = conv1 + gux[c][j] * (u[j] - w[j])
                        convn = convn + -(w[j] - un[j]) * guxn[c][j]
                    val = ((u[c] * J - un[c] * Jn) * idt - divw1 * J * u[c] * 0.5 - divwn * (Jn * un[c]) * 0.5
                           + conv1 * J * 0.5 + convn * Jn * 0.5)
                    add_rows(rows_c, val * (prob.rho_f * wq), Nb)
                    for k in range(n):
                        Tk = sig[c][0] * Finv[k][0]
                        Tkn = sign[c][0] * Finvn[k][0]
                        for j in range(1, n):
                            Tk = Tk + sig[c][j] * Finv[k][j]
                            Tkn = Tkn + sign[c][j] * Finvn[k][j]
                        add_rows(rows_c, (Tk * J * 0.5 + Tkn * Jn * 0.5) * wq, Gh[:, :, k])
                else:
                    conv = gux[c][0] * adv[0]
                    for j in range(1, n):
                        conv = conv + gux[c][j] * adv[j]
                    if bdf:
                        conv = conv + ut[c]
                    add_rows(rows_c, conv * J * (prob.rho_f * wq), Nb)
                    for k in range(n):
                        Tk = sig[c][0] * Finv[k][0]
                        for j in range(1, n):
                            Tk = Tk + sig[c][j] * Finv[k][j]
                        add_rows(rows_c, Tk * J * wq, Gh[:, :, k])
                arow = np.where(ale_rows >= 0, ale_rows + c, -1)
                for j in range(n):
                    if prob.ale_op == 0:
                        t = (gd[c][j] + gd[j][c]) * (kale * wq)
                    else:
                        t = gd[c][j] * (kale * wq)
                    add_rows(arow, t, Gh[:, :, j])
            mass = J * div
        prow = nd * nloc + np.arange(dim + 1)
        add_rows(prow, mass * wq, np.broadcast_to(psi[None, :], (E, dim + 1)))
        if source is not None:
            xq = lo + (np.array(xi)[None, :] + 1.0) * 0.5 * h
            fm, gm, ga = source(xq)
            ee = np.arange(E)[:, None]
            for c in range(n):
                rows = (np.where(iface, a_idx[None, :] * nd, a_idx[None, :] * nd + n) if not solid
                        else a_idx[None, :] * nd + np.zeros((E, 1), dtype=np.int64)) + c
                rho = prob.rho_s if solid else prob.rho_f
                Rv[ee, rows] -= (rho * fm[:, c] * wq)[:, None] * Nb
                if ga is not None and not solid:
                    arow = np.where(iface, -1, a_idx[None, :] * nd + c)
                    sel = arow >= 0
                    contrib = (ga[:, c] * wq)[:, None] * Nb
                    np.subtract.at(Rv, (np.nonzero(sel)[0], arow[sel]), contrib[sel])
            Rv[:, prow] -= (gm * wq)[:, None] * psi[None, :]
    return Rv, Rg


def _solid_piola(prob, F, Finv, J, p, n):
    """First Piola stress P = J sigma F^{-T} of the incompressible solid
    (Sec. 2.2): -p J F^{-T} + 2 C1 J F - 2 C2 J F^{-T} F^{-1} F^{-T} with
    2 C1 = mu_s - 2 C2 (C2 = 0: Neo-Hookean); entries are Duals or arrays."""
    c2 = getattr(prob, "mr_c2", 0.0)
    pJ = p * J
    muJ = J * (prob.mu_s - 2.0 * c2)                # 2 C1 J
    T = [[-(pJ * Finv[j][i]) + muJ * F[i][j] for j in range(n)] for i in range(n)]
    if c2 != 0.0:
        # Q = F^{-1} F^{-T} (Q_ab = sum_m Finv_am Finv_bm), (F^{-T} Q)_ij = sum_a Finv_ai Q_aj
        Q = [[None] * n for _ in range(n)]
        for a_ in range(n):
            for b_ in range(n):
                q_ = Finv[a_][0] * Finv[b_][0]
                for m_ in range(1, n):
                    q_ = q_ + Finv[a_][m_] * Finv[b_][m_]
                Q[a_][b_] = q_
        c2J = J * (2.0 * c2)
        for i in range(n):
            for j in range(n):
                g_ = Finv[0][i] * Q[0][j]
                for a_ in range(1, n):
                    g_ = g_ + Finv[a_][i] * Q[a_][j]
                T[i][j] = T[i][j] - c2J * g_
    return T


def fe_pattern(lev: Level) -> sp.csr_matrix:
    """Full FE graph (Sec. 3.1 blocks): node-node unknowns of nodes sharing an
    element, node-pressure and pressure-node within an element, no
    pressure-pressure.  Columns sorted; all values zero."""
    nd = 2 * lev.dim
    nn = nd * 3 ** lev.dim
    rows, cols = [], []
    ed = lev.elem_dofs
    for i in range(ed.shape[1]):
        for j in range(ed.shape[1]):
            if i >= nn and j >= nn:
                continue
            rows.append(ed[:, i])
            cols.append(ed[:, j])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    A = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(lev.N, lev.N))
    A.sum_duplicates()
    A.sort_indices()
    A.data[:] = 0.0
    return A


def place_on_pattern(pattern: sp.csr_matrix, M: sp.spmatrix) -> sp.csr_matrix:
    """Values of M on the given pattern (M's entries must lie inside it)."""
    M = sp.coo_matrix(M)
    P = pattern.tocoo()
    N = pattern.shape[1]
    pk = P.row.astype(np.int64) * N + P.col
    mk = M.row.astype(np.int64) * N + M.col
    order = np.argsort(pk)
    pos = np.searchsorted(pk[order], mk)
    pos = np.minimum(pos, len(pk) - 1)
    ok = pk[order][pos] == mk
    if not np.all(ok | (M.data == 0.0)):
        raise ValueError("matrix entries outside the FE pattern")
    data = np.zeros(len(pk))
    np.add.at(data, order[pos[ok]], M.data[ok])
    out = pattern.copy()
    # pattern is csr with sorted indices; coo order of P equals csr order
    out.data = data
    return out


def inflow_alpha(t: float) -> float:
    """Pulsating inflow amplitude of the transient workload."""
    return 0.5 * (1.0 + np.sin(2.0 * np.pi * t))


def assemble(prob, lev: Level, y: np.ndarray, source=None, chunk: int = 2048, tr: Optional[dict] = None):
    """Global residual r(y) and exact Jacobian J(y) (CSR on the FE pattern),
    Dirichlet rows replaced by identity rows (Sec. 2.3 / 3.1).  With ``tr``
    (transient) the Dirichlet data are those at time tr["t"]."""
    r = np.zeros(lev.N)
    rows_all, cols_all, vals_all = [], [], []
    nd = 2 * lev.dim
    nn = nd * 3 ** lev.dim
    for solid in (True, False):
        elems_all = np.nonzero(lev.elem_solid == solid)[0]
        for s in range(0, len(elems_all), chunk):
            elems = elems_all[s:s + chunk]
            Rv, Rg = element_system(prob, lev, elems, y, source, tr)
            ed = lev.elem_dofs[elems]
            np.add.at(r, ed, Rv)
            m = ed.shape[1]
            keep = np.ones((m, m), dtype=bool)
            keep[nn:, nn:] = False
            assert np.all(Rg[:, ~keep] == 0.0)
            ii, jj = np.nonzero(keep)
            rows_all.append(ed[:, ii].reshape(-1))
            cols_all.append(ed[:, jj].reshape(-1))
            vals_all.append(Rg[:, ii, jj].reshape(-1))
    Jc = sp.coo_matrix((np.concatenate(vals_all), (np.concatenate(rows_all), np.concatenate(cols_all))),
                       shape=(lev.N, lev.N))
    J = place_on_pattern(fe_pattern(lev), Jc)
    apply_dirichlet_rows(J, lev.dir_mask)
    alpha = 1.0 if tr is None else inflow_alpha(tr["t"])
    r[lev.dir_mask] = y[lev.dir_mask] - alpha * lev.dir_val[lev.dir_mask]
    return r, J


def apply_dirichlet_rows(J: sp.csr_matrix, mask: np.ndarray) -> None:
    """Row i := e_i^T for every Dirichlet unknown i (pattern kept)."""
    for i in np.nonzero(mask)[0]:
        a, b = J.indptr[i], J.indptr[i + 1]
        J.data[a:b] = 0.0
        k = a + np.searchsorted(J.indices[a:b], i)
        J.data[k] = 1.0


def residual_only(prob, lev: Level, y: np.ndarray, source=None, tr=None) -> np.ndarray:
    return assemble(prob, lev, y, source, tr=tr)[0]


def bdf_coefficients(order: int):
    """BDF time-derivative coefficients (a0, a1, a2) of q^{n+1}, q^n, q^{n-1}."""
    return (1.0, -1.0, 0.0) if order == 1 else (1.5, -2.0, 0.5)
