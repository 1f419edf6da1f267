"""Pins of the oracle's mesh / numbering / patch definitions (CPU only)."""
import os

import numpy as np
import pytest

from oracle.mesh import (FLUID, IFACE, SOLID, build_level, build_patches, initial_state,
                         n_unknowns)
from paper_1709_05660_gb300.workloads import CONFIGS, Problem, noise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_paper_3d_unknown_counts():
    """Sec. 4 table of 3D unknowns == Q2-P1disc count of the refined 8x2x2 box."""
    got = 0
    for row in _golden():
        if row[0] != "3d":
            continue
        level, count = int(row[1]), int(row[2])
        s = 2 ** (level - 1)
        assert n_unknowns(3, (8 * s, 2 * s, 2 * s)) == count
        got += 1
    assert got == 5


def test_mesh_count_matches_closed_form():
    box = Problem(dim=3, breaks=(tuple(np.linspace(0, 1.5, 9)), (0.0, 0.2, 0.4), (0.0, 0.2, 0.4)),
                  levels=2, flap_lo=(0.5, 0.0, 0.1), flap_hi=(0.55, 0.25, 0.4))
    for l in range(2):
        lev = build_level(box, l)
        assert lev.N == n_unknowns(3, lev.cells)
    assert build_level(box, 1).N == 17062   # level 2 of the paper's 3D table
    p, _ = CONFIGS["channel2d_l3"]
    lev = build_level(p, 2)
    assert lev.cells == (64, 16) and lev.n_nodes == 4257 and lev.N == 20100


def test_paper_block_sizes():
    """Sec. 3.3: 16-element (2D) / 64-element (3D) blocks hold 372 / 4630 unknowns."""
    want = {r[1]: int(r[3]) for r in _golden() if r[0] == "block"}
    p2 = Problem(breaks=(tuple(np.linspace(0, 2, 9)), tuple(np.linspace(0, 1, 9))), levels=1,
                 flap_lo=(5, 5), flap_hi=(6, 6))
    lev = build_level(p2, 0)
    pts = build_patches(lev, (4, 4))
    assert len(pts) == 4 and all(len(pt.dofs) == want["2d"] for pt in pts)
    p3 = Problem(dim=3, breaks=(tuple(np.linspace(0, 1, 5)),) * 3, levels=1,
                 flap_lo=(5, 5, 5), flap_hi=(6, 6, 6))
    lev3 = build_level(p3, 0)
    pts3 = build_patches(lev3, (4, 4, 4))
    assert len(pts3) == 1 and len(pts3[0].dofs) == want["3d"]


@pytest.mark.parametrize("cfg", ["channel2d_l3"])
def test_patches_partition_and_materials(cfg):
    prob, opts = CONFIGS[cfg]
    for l in range(1, prob.levels):
        lev = build_level(prob, l)
        pts = build_patches(lev, opts.tile)
        count = np.zeros(lev.N, dtype=np.int64)
        for pt in pts:
            assert len(np.unique(lev.elem_solid[pt.elems])) == 1          # never straddles
            count[pt.dofs[pt.owned]] += 1
            nd = 2 * lev.dim
            nn = lev.n_nodes * nd
            nodes = np.unique(pt.dofs[pt.dofs < nn] // nd)
            assert set(nodes) == set(lev.elem_nodes[pt.elems].reshape(-1))  # closure rule
            if not pt.solid:
                own_nodes = pt.dofs[pt.owned & (pt.dofs < nn)] // nd
                assert np.all(lev.node_class[own_nodes] != IFACE)        # interface -> solid blocks
        assert np.all(count == 1)                                         # R^0 partition


def test_node_classes_and_dirichlet():
    prob, _ = CONFIGS["channel2d_l3"]
    lev = build_level(prob, 0)
    # flap = coarse x cell 4, y cells 0-1: 2 solid elements, interface nodes on its 3 free sides
    assert lev.elem_solid.sum() == 2
    iface = np.nonzero(lev.node_class == IFACE)[0]
    xy = lev.node_xyz[iface]
    on_left = np.isclose(xy[:, 0], 0.5) & (xy[:, 1] <= 0.25 + 1e-12)
    on_right = np.isclose(xy[:, 0], 0.55) & (xy[:, 1] <= 0.25 + 1e-12)
    on_top = np.isclose(xy[:, 1], 0.25) & (xy[:, 0] >= 0.5 - 1e-12) & (xy[:, 0] <= 0.55 + 1e-12)
    assert np.all(on_left | on_right | on_top)
    assert len(iface) == 5 + 5 + 1       # 5 nodes per vertical side, 1 top midpoint
    # outflow: d fixed, u free (except wall corners)
    nd = 4
    out = np.nonzero(np.isclose(lev.node_xyz[:, 0], 2.0))[0]
    assert np.all(lev.dir_mask[out * nd]) and np.all(lev.dir_mask[out * nd + 1])
    mid = out[(lev.node_xyz[out, 1] > 0) & (lev.node_xyz[out, 1] < 0.5)]
    assert not np.any(lev.dir_mask[mid * nd + 2])
    # inflow parabola has mean U (Simpson on the 9 nodes is exact for a parabola)
    inl = np.nonzero(np.isclose(lev.node_xyz[:, 0], 0.0))[0]
    vals = lev.dir_val[inl * nd + 2]
    ys = lev.node_xyz[inl, 1]
    order = np.argsort(ys)
    h = 0.0625
    simpson = h / 3 * (vals[order][0] + vals[order][-1] + 4 * vals[order][1:-1:2].sum()
                       + 2 * vals[order][2:-1:2].sum())
    assert simpson / 0.5 == pytest.approx(prob.U, rel=1e-12)


def test_initial_state_recipe():
    prob, _ = CONFIGS["channel2d_l3"]
    lev = build_level(prob, 2)
    nz = noise(lev.N, 0)
    y = initial_state(prob, lev, nz)
    assert np.all(y[lev.dir_mask] == lev.dir_val[lev.dir_mask])
    nd = 4
    dfree = np.zeros(lev.N, dtype=bool)
    dfree[0:lev.n_nodes * nd:nd] = True
    dfree[1:lev.n_nodes * nd:nd] = True
    dfree &= ~lev.dir_mask
    assert np.all(y[dfree] == nz[dfree])
    assert np.all(y[lev.n_nodes * nd:] == 0.0)
    solid_u = np.nonzero(lev.node_class != FLUID)[0] * nd + 2
    assert np.all(y[solid_u][~lev.dir_mask[solid_u]] == 0.0)
