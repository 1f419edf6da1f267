"""Launch shapes (fsi_set_launch_params) and their autotuner on the device.

The 3-level 2D channel (20,100 unknowns), mixed path.  Forcing any candidate shape (one block per
Schwarz block or row slices with several column-group counts, 2 / 4 / 8
threads per SpMV row, panel width 16 or 32) changes only the rounding order:
the V-cycle matches the built-in shapes to FP32 rounding, and the Newton
correction stays within the mixed path's 1e-8 of the oracle's direct
solution.  The tuner's entry passes the table checks and solves to the same
bar.  Bad values and timing before a factorisation are rejected.
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


@pytest.fixture(scope="module")
def case():
    prob, opts = CONFIGS["channel2d_l3"]
    opts = replace(opts, precision=1)
    orc = osolver.Oracle(prob, opts)
    y0 = initial_state(prob, orc.fine, noise(orc.fine.N, 0))
    r, J = orc.assemble(y0)
    xs = osolver.direct_solve(J, -r)
    return dict(prob=prob, opts=opts, y0=y0, xs=xs, N=orc.fine.N)


def _instance(case):
    from paper_1709_05660_gb300 import fsi
    s = fsi.FSI(case["prob"], case["opts"], stream=torch.cuda.current_stream().cuda_stream, tuned=False)
    s.set_state(_dev(case["y0"]))
    s.assemble()
    s.factor()
    return s


def _vcycle(s, b):
    z = torch.empty_like(b)
    s.apply_vcycle(b, z)
    return z.cpu().numpy()


def _newton_err(s, case):
    dx = torch.empty(case["N"], dtype=torch.float64, device="cuda")
    s.set_state(_dev(case["y0"]))
    _, st = s.newton_step(dx)
    return np.linalg.norm(dx.cpu().numpy() - case["xs"]) / np.linalg.norm(case["xs"]), st.iters


SHAPES = [dict(apply_slices=1), dict(apply_slices=3, apply_groups=8), dict(apply_slices=8, apply_groups=32),
          dict(apply_slices=2, apply_groups=4, spmv_sub=2), dict(apply_slices=16, apply_groups=16, spmv_sub=8)]


@pytest.mark.parametrize("shape", SHAPES, ids=[str(i) for i in range(len(SHAPES))])
def test_forced_shapes_change_rounding_only(case, shape):
    s = _instance(case)
    try:
        L = case["prob"].levels
        b = _dev(np.random.default_rng(1).standard_normal(case["N"]))
        z0 = _vcycle(s, b)
        _, it0 = _newton_err(s, case)
        for l in range(1, L):
            s.set_launch_params(l, **shape)
            got = s.get_launch_params(l)
            if shape.get("apply_slices") == 1:
                assert got["apply_slices"] == 1
            else:
                assert 2 <= got["apply_slices"] <= shape["apply_slices"]
                assert 1 <= got["apply_groups"] <= shape["apply_groups"]
            assert got["spmv_sub"] == shape.get("spmv_sub", 4)
        z = _vcycle(s, b)
        assert np.linalg.norm(z - z0) <= 1e-5 * np.linalg.norm(z0)
        err, it = _newton_err(s, case)
        assert err <= 1e-8, err
        assert abs(it - it0) <= 1
    finally:
        s.close()


@pytest.mark.parametrize("panel", [16, 32, 216])
def test_panel_width(case, panel):
    s = _instance(case)
    try:
        L = case["prob"].levels
        s.set_launch_params(L - 1, gj_panel=panel)
        assert s.get_launch_params(L - 1)["gj_panel"] == panel
        err, _ = _newton_err(s, case)   # refactors with the chosen panel width
        assert err <= 1e-8, err
    finally:
        s.close()


def test_tuner_entry_is_valid_and_solves(case):
    from paper_1709_05660_gb300 import autotune, fsi
    entry = autotune.tune(case["prob"], case["opts"], stream=torch.cuda.current_stream().cuda_stream, reps=5,
                          trials=1, log=lambda m: None)
    autotune.check_entry(entry, case["prob"].levels)
    assert entry["gj_panel"] in autotune.PANEL_CANDIDATES
    s = fsi.FSI(case["prob"], case["opts"], stream=torch.cuda.current_stream().cuda_stream, tuned=False)
    try:
        assert autotune.apply_table(s, entry) is entry
        for l in range(1, case["prob"].levels):
            got = s.get_launch_params(l)
            assert got["apply_slices"] == entry["levels"][str(l)]["apply_slices"]
            assert got["spmv_sub"] == entry["levels"][str(l)]["spmv_sub"]
        err, _ = _newton_err(s, case)
        assert err <= 1e-8, err
    finally:
        s.close()


def test_rejects_bad_values_and_timing_before_factor(case):
    from paper_1709_05660_gb300 import fsi
    s = fsi.FSI(case["prob"], case["opts"], stream=torch.cuda.current_stream().cuda_stream, tuned=False)
    try:
        with pytest.raises(fsi.FSIError):
            s.time_level_kernels(1, 10)                      # no factorisation yet
        for bad in (dict(spmv_sub=3), dict(gj_panel=20), dict(apply_slices=-1), dict(apply_groups=1000)):
            with pytest.raises(fsi.FSIError):
                s.set_launch_params(1, **bad)
        with pytest.raises(fsi.FSIError):
            s.set_launch_params(0, apply_slices=2)           # level 0 has no Schwarz blocks
        s.set_state(_dev(case["y0"]))
        s.assemble()
        s.factor()
        a, m = s.time_level_kernels(case["prob"].levels - 1, 3)
        assert a > 0 and m > 0
    finally:
        s.close()
