"""CPU checks of libfsi's host logic (no GPU): the library loads and exports
every function include/fsi.h declares, and the host-only plan of a hierarchy
(numbering, FE pattern, node classes, Dirichlet data, Schwarz blocks, grid
transfers) is bit-identical to the oracle's."""
import os
import re
from dataclasses import replace

import numpy as np
import pytest

from oracle import fem, solver
from oracle.mesh import build_level, build_patches
from paper_1709_05660_gb300.workloads import CONFIGS, SolverOpts
from tests.oracle_cases import SMALL_3D, UNIT_FLUID

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_05660_gb300 import build, fsi
    if not os.path.exists(fsi.LIB_PATH):
        build.build()
    return fsi


def test_library_exports_header_symbols(lib):
    hdr = open(os.path.join(ROOT, "include", "fsi.h")).read()
    names = set(re.findall(r"^\s*(?:int|void|const char\*|int64_t)\s+(fsi_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 20
    L = lib.load_library()
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert names <= set(lib.SYMBOLS)


def _plan(lib, prob, opts):
    return lib.FSI(prob, opts, plan_only=True)


PLAN_CASES = {
    "c1": lambda: CONFIGS["channel2d_l3"],
    "3d": lambda: (replace(SMALL_3D, levels=2), SolverOpts(tile=(2, 2, 2))),
    # ragged blocks: 3 x 3 tiles do not divide the 64 x 16 fine mesh, and they are split by material
    "ragged_tile": lambda: (CONFIGS["channel2d_l3"][0], SolverOpts(tile=(3, 3))),
    # a tile larger than the mesh: one block per material region
    "tile_beyond_mesh": lambda: (replace(CONFIGS["channel2d_l3"][0], levels=2), SolverOpts(tile=(100, 100))),
    # one level: coarse operator only, no Schwarz level
    "one_level": lambda: (replace(CONFIGS["channel2d_l3"][0], levels=1), SolverOpts(tile=(2, 2))),
    # no solid and no interface (the flap box lies outside the domain)
    "all_fluid": lambda: (replace(UNIT_FLUID, levels=2), SolverOpts(tile=(2, 2))),
    # ragged 3D blocks
    "3d_ragged": lambda: (replace(SMALL_3D, levels=2), SolverOpts(tile=(3, 2, 3))),
}


@pytest.mark.parametrize("case", list(PLAN_CASES))
def test_plan_matches_oracle_bit_exact(lib, case):
    prob, opts = PLAN_CASES[case]()
    s = _plan(lib, prob, opts)
    for l in range(prob.levels):
        lev = build_level(prob, l)
        assert int(s.N[l]) == lev.N
        # FE pattern
        rowptr, col, _ = s.export_csr(l, values=False)
        pat = fem.fe_pattern(lev)
        assert np.array_equal(rowptr, pat.indptr.astype(np.int64))
        assert np.array_equal(col, pat.indices.astype(np.int32))
        assert int(s.nnz[l]) == pat.nnz
        # classes, materials, Dirichlet data
        nc, es, dm, dv = s.export_dofmap(l, lev.n_nodes, lev.n_elem)
        assert np.array_equal(nc, lev.node_class.astype(np.uint8))
        assert np.array_equal(es.astype(bool), lev.elem_solid)
        assert np.array_equal(dm, lev.dir_mask)
        assert np.array_equal(dv, lev.dir_val)
        if l == 0:
            continue
        # Schwarz blocks
        pts = build_patches(lev, opts.tile)
        got = s.export_patches(l)
        assert len(got) == len(pts)
        for (dofs, owned), pt in zip(got, pts):
            assert np.array_equal(dofs, pt.dofs.astype(np.int32))
            assert np.array_equal(owned, pt.owned)
        # transfers
        coarse = build_level(prob, l - 1)
        P, R = solver.transfer_operators(coarse, lev)
        for which, M in ((0, P), (1, R)):
            M = M.tocsr()
            M.sort_indices()
            rp, c, v = s.export_transfer(l, which)
            assert np.array_equal(rp, M.indptr.astype(np.int64))
            assert np.array_equal(c, M.indices.astype(np.int32))
            assert np.array_equal(v, M.data)
    s.close()


def test_plan_sizes_5level_channel_and_3d_counts(lib):
    prob, opts = CONFIGS["channel2d_l5"]
    s = _plan(lib, prob, opts)
    assert int(s.N[-1]) == 313860
    s.close()


def test_compute_on_planned_ctx_is_rejected(lib):
    prob, opts = CONFIGS["channel2d_l3"]
    s = _plan(lib, prob, opts)
    y = np.zeros(int(s.N[-1]))
    with pytest.raises(lib.FSIError) as ei:
        s.set_state(y)
    assert ei.value.code == -1
    s.close()


def test_invalid_descriptors_rejected(lib):
    prob, opts = CONFIGS["channel2d_l3"]
    with pytest.raises(lib.FSIError):
        _plan(lib, replace(prob, levels=0), opts)
    with pytest.raises(lib.FSIError):
        _plan(lib, prob, replace(opts, restart=0))
    with pytest.raises(lib.FSIError):
        _plan(lib, replace(prob, breaks=((0.0, 1.0, 0.5), prob.breaks[1])), opts)


def test_initial_state_on_a_planned_ctx_is_bit_exact():
    """fsi_initial_state is a host computation: a planned ctx (no GPU) gives
    the oracle's benchmark state bit for bit, and with zero noise the
    boundary-condition lift that starts a nonlinear solve."""
    from oracle.mesh import build_level, initial_state
    from paper_1709_05660_gb300 import fsi
    from paper_1709_05660_gb300.workloads import CONFIGS, noise, problem_3d
    for prob, opts in (CONFIGS["channel2d_l3"], (problem_3d(levels=1), CONFIGS["box3d_l3_bdf2"][1])):
        p = fsi.FSI(prob, opts, plan_only=True)
        N = int(p.N[-1])
        lev = build_level(prob, prob.levels - 1)
        for nz in (noise(N, 0), np.zeros(N)):
            y = np.empty(N)
            p.initial_state(nz, y)
            assert np.array_equal(y, initial_state(prob, lev, nz))
        p.close()
