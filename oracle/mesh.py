"""Oracle: mesh hierarchy, unknown numbering, node classes, Dirichlet data and
Schwarz patches.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed:

* Mesh hierarchy by midpoint refinement of a conforming coarse mesh
  (Sec. 3.2); the fluid-solid interface lies on element edges (Sec. 2.5).
* Q2 (continuous, 3^n nodes per element) displacement and velocity, P1disc
  pressure with n+1 unknowns per element (Sec. 2.5).
* Unknown vector y = (d, u, p) (Sec. 3.1).  Numbering: Q2 nodes
  lexicographic (x fastest); node unknown = node*2n + c with
  c in [d_0..d_{n-1}, u_0..u_{n-1}]; pressures follow all node unknowns,
  element-lexicographic, then k in {1, xi, eta(, zeta)}.
* Node classes s / i / f of Sec. 3.1: a node touching only solid elements is
  solid, only fluid elements is fluid, both is an interface node.
* Schwarz subdomains (Sec. 3.3): aligned tiles of elements split by material
  so that no block straddles the interface; the overlapping set R^delta_k is
  every d,u unknown on the closure of the block's elements plus their
  pressures (this reproduces the 372 / 4630 unknowns per 16 / 64-element
  block printed in Sec. 3.3); the owned set R^0_k gives each node to the
  block of the lowest-numbered element containing it, solid elements first.
"""
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

FLUID, SOLID, IFACE = 0, 1, 2


def n_unknowns(dim: int, cells: Tuple[int, ...]) -> int:
    """Closed-form Q2-P1disc unknown count on a tensor mesh (Sec. 4, Table 1)."""
    nodes = 1
    elems = 1
    for c in cells:
        nodes *= 2 * c + 1
        elems *= c
    return 2 * dim * nodes + (dim + 1) * elems


def refine_breaks(breaks: np.ndarray, times: int) -> np.ndarray:
    """Midpoint refinement of a 1D vertex list (Sec. 3.2)."""
    v = np.asarray(breaks, dtype=np.float64)
    for _ in range(times):
        mid = (v[:-1] + v[1:]) / 2.0
        w = np.empty(2 * len(v) - 1)
        w[0::2] = v
        w[1::2] = mid
        v = w
    return v


def q2_coords(vertices: np.ndarray) -> np.ndarray:
    """Q2 node coordinates along one axis: vertices and cell midpoints."""
    q = np.empty(2 * len(vertices) - 1)
    q[0::2] = vertices
    q[1::2] = (vertices[:-1] + vertices[1:]) / 2.0
    return q


@dataclass
class Level:
    dim: int
    cells: Tuple[int, ...]          # elements per axis
    verts: List[np.ndarray]         # vertex coordinates per axis
    nodes_ax: Tuple[int, ...]       # Q2 nodes per axis
    coords: List[np.ndarray]        # Q2 node coordinates per axis
    n_nodes: int
    n_elem: int
    N: int
    elem_nodes: np.ndarray          # (E, 3^dim) global node ids
    elem_solid: np.ndarray          # (E,) bool
    elem_lo: np.ndarray             # (E, dim) lower corner
    elem_h: np.ndarray              # (E, dim) edge lengths
    node_class: np.ndarray          # (Nn,) FLUID / SOLID / IFACE
    node_xyz: np.ndarray            # (Nn, dim)
    elem_dofs: np.ndarray           # (E, 2n*3^n + n+1) global unknowns
    dir_mask: np.ndarray            # (N,) bool
    dir_val: np.ndarray             # (N,) float64

    @property
    def nd_node(self) -> int:
        return 2 * self.dim

    def pressure_dof(self, e: int, k: int) -> int:
        return self.n_nodes * 2 * self.dim + e * (self.dim + 1) + k


def _lex(idx: Tuple[int, ...], ext: Tuple[int, ...]) -> int:
    out = 0
    stride = 1
    for i, n in zip(idx, ext):
        out += i * stride
        stride *= n
    return out


def inflow_profile(prob, xyz: np.ndarray, U: float) -> np.ndarray:
    """Inflow x-velocity (Sec. 4): parabola 1.5 U y(H-y)/(H/2)^2 in 2D.

    3D: the product parabola 36 U y(H_y-y) z(H_z-z) / (H_y^2 H_z^2) (mean U),
    an adaptation of the 3D profile of Sec. 4 to a channel walled on four
    sides.
    """
    Hy = prob.breaks[1][-1]
    y = xyz[..., 1]
    if prob.dim == 2:
        return 1.5 * U * y * (Hy - y) / (Hy / 2.0) ** 2
    Hz = prob.breaks[2][-1]
    z = xyz[..., 2]
    return 36.0 * U * y * (Hy - y) * z * (Hz - z) / (Hy * Hy * Hz * Hz)


def build_level(prob, l: int) -> Level:
    dim = prob.dim
    verts = [refine_breaks(np.asarray(b), l) for b in prob.breaks]
    cells = tuple(len(v) - 1 for v in verts)
    coords = [q2_coords(v) for v in verts]
    nodes_ax = tuple(len(c) for c in coords)
    n_nodes = int(np.prod(nodes_ax))
    n_elem = int(np.prod(cells))
    N = 2 * dim * n_nodes + (dim + 1) * n_elem
    nloc = 3 ** dim

    # element -> nodes, geometry and material (centroid in the flap box)
    elem_nodes = np.zeros((n_elem, nloc), dtype=np.int64)
    elem_lo = np.zeros((n_elem, dim))
    elem_h = np.zeros((n_elem, dim))
    elem_solid = np.zeros(n_elem, dtype=bool)
    for e in range(n_elem):
        ei = []
        r = e
        for c in cells:
            ei.append(r % c)
            r //= c
        for a in range(nloc):
            li = []
            r = a
            for _ in range(dim):
                li.append(r % 3)
                r //= 3
            elem_nodes[e, a] = _lex(tuple(2 * ei[d] + li[d] for d in range(dim)), nodes_ax)
        inside = True
        for d in range(dim):
            lo, hi = verts[d][ei[d]], verts[d][ei[d] + 1]
            elem_lo[e, d] = lo
            elem_h[e, d] = hi - lo
            cen = 0.5 * (lo + hi)
            inside &= (prob.flap_lo[d] < cen < prob.flap_hi[d])
        elem_solid[e] = inside

    touch_s = np.zeros(n_nodes, dtype=bool)
    touch_f = np.zeros(n_nodes, dtype=bool)
    for e in range(n_elem):
        if elem_solid[e]:
            touch_s[elem_nodes[e]] = True
        else:
            touch_f[elem_nodes[e]] = True
    node_class = np.where(touch_s & touch_f, IFACE, np.where(touch_s, SOLID, FLUID)).astype(np.int8)

    # node coordinates
    node_xyz = np.zeros((n_nodes, dim))
    grids = np.meshgrid(*coords, indexing="ij")
    for d in range(dim):
        # lexicographic with x fastest == Fortran order of an (nx, ny, nz) grid
        node_xyz[:, d] = grids[d].reshape(-1, order="F")

    nd = 2 * dim
    elem_dofs = np.zeros((n_elem, nd * nloc + dim + 1), dtype=np.int64)
    for a in range(nloc):
        for s in range(nd):
            elem_dofs[:, a * nd + s] = elem_nodes[:, a] * nd + s
    for k in range(dim + 1):
        elem_dofs[:, nd * nloc + k] = n_nodes * nd + np.arange(n_elem) * (dim + 1) + k

    # Dirichlet data: d = 0 on the whole outer boundary; u Dirichlet on the
    # inflow and the walls (profile at the inflow, no-slip on walls, which
    # also clamps the flap at y = 0); the outflow x = L is stress-free.
    dir_mask = np.zeros(N, dtype=bool)
    dir_val = np.zeros(N)
    ijk = np.zeros((n_nodes, dim), dtype=np.int64)
    r = np.arange(n_nodes)
    for d in range(dim):
        ijk[:, d] = r % nodes_ax[d]
        r = r // nodes_ax[d]
    on_bnd = np.zeros(n_nodes, dtype=bool)
    on_wall_or_in = ijk[:, 0] == 0
    for d in range(dim):
        on_bnd |= (ijk[:, d] == 0) | (ijk[:, d] == nodes_ax[d] - 1)
        if d > 0:
            on_wall_or_in |= (ijk[:, d] == 0) | (ijk[:, d] == nodes_ax[d] - 1)
    for c in range(dim):
        dir_mask[np.nonzero(on_bnd)[0] * nd + c] = True
    for c in range(dim):
        dir_mask[np.nonzero(on_wall_or_in)[0] * nd + dim + c] = True
    inflow_nodes = np.nonzero(ijk[:, 0] == 0)[0]
    dir_val[inflow_nodes * nd + dim] = inflow_profile(prob, node_xyz[inflow_nodes], prob.U)

    return Level(dim=dim, cells=cells, verts=verts, nodes_ax=nodes_ax, coords=coords,
                 n_nodes=n_nodes, n_elem=n_elem, N=N, elem_nodes=elem_nodes,
                 elem_solid=elem_solid, elem_lo=elem_lo, elem_h=elem_h,
                 node_class=node_class, node_xyz=node_xyz, elem_dofs=elem_dofs,
                 dir_mask=dir_mask, dir_val=dir_val)


def build_hierarchy(prob) -> List[Level]:
    return [build_level(prob, l) for l in range(prob.levels)]


def initial_state(prob, lev: Level, noise: np.ndarray) -> np.ndarray:
    """Benchmark linearisation state (synthetic stand-in for a Newton iterate).

    d = 0 and p = 0; u_x = inflow profile at every fluid node with a free
    u_x, 0 at interface and solid nodes; Dirichlet values at Dirichlet
    unknowns; then ``noise`` is added at every free displacement unknown.
    """
    dim, nd = lev.dim, 2 * lev.dim
    y = np.zeros(lev.N)
    fluid_nodes = np.nonzero(lev.node_class == FLUID)[0]
    ux = fluid_nodes * nd + dim
    y[ux] = inflow_profile(prob, lev.node_xyz[fluid_nodes], prob.U)
    y[lev.dir_mask] = lev.dir_val[lev.dir_mask]
    dmask = np.zeros(lev.N, dtype=bool)
    for c in range(dim):
        dmask[np.arange(lev.n_nodes) * nd + c] = True
    dmask &= ~lev.dir_mask
    y[dmask] += noise[: lev.N][dmask]
    return y


@dataclass
class Patch:
    elems: np.ndarray     # element ids
    dofs: np.ndarray      # R^delta_k, ascending global unknowns
    owned: np.ndarray     # bool per entry of dofs (R^0_k)
    solid: bool


def node_owner_elements(lev: Level) -> np.ndarray:
    """Element that owns each node: lowest-numbered containing element,
    solid elements ranked before fluid ones (Sec. 3.3 reading)."""
    owner = -np.ones(lev.n_nodes, dtype=np.int64)
    order = list(np.nonzero(lev.elem_solid)[0]) + list(np.nonzero(~lev.elem_solid)[0])
    for e in order:
        nodes = lev.elem_nodes[e]
        free = owner[nodes] < 0
        owner[nodes[free]] = e
    return owner


def build_patches(lev: Level, tile: Tuple[int, ...]) -> List[Patch]:
    """Schwarz blocks of Sec. 3.3 for one level."""
    dim, nd = lev.dim, 2 * lev.dim
    ntile = tuple((c + t - 1) // t for c, t in zip(lev.cells, tile))
    key_of_elem = np.zeros(lev.n_elem, dtype=np.int64)
    for e in range(lev.n_elem):
        r = e
        tid = []
        for c, t in zip(lev.cells, tile):
            tid.append((r % c) // t)
            r //= c
        key_of_elem[e] = _lex(tuple(tid), ntile) * 2 + (0 if lev.elem_solid[e] else 1)
    keys = np.unique(key_of_elem)
    patch_of_elem = np.searchsorted(keys, key_of_elem)
    owner_elem = node_owner_elements(lev)
    patches: List[Patch] = []
    for k, key in enumerate(keys):
        elems = np.nonzero(key_of_elem == key)[0]
        nodes = np.unique(lev.elem_nodes[elems].reshape(-1))
        node_dofs = (nodes[:, None] * nd + np.arange(nd)[None, :]).reshape(-1)
        p_dofs = (lev.n_nodes * nd + elems[:, None] * (dim + 1) + np.arange(dim + 1)[None, :]).reshape(-1)
        dofs = np.concatenate([node_dofs, p_dofs])
        own_node = np.repeat(patch_of_elem[owner_elem[nodes]] == k, nd)
        owned = np.concatenate([own_node, np.ones(len(p_dofs), dtype=bool)])
        order = np.argsort(dofs, kind="stable")
        patches.append(Patch(elems=elems, dofs=dofs[order], owned=owned[order],
                             solid=bool(key % 2 == 0)))
    return patches
