"""Nested iteration (full multigrid) for the steady problem on the device
(fsi_fmg_newton) against the oracle's fmg_newton on the 3-level channel:
the same Newton step count on every mesh level (within 1) and the same
finest steady state (both end with Newton steps below 1e-10 of ||y||, so the
states agree far below 1e-8)."""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import solver as osolver  # noqa: E402
from paper_1709_05660_gb300.workloads import Problem, SolverOpts  # noqa: E402

PROB = Problem(levels=3, mu_s=5e5, U=0.2)


@pytest.fixture(scope="module")
def oracle_fmg():
    return osolver.fmg_newton(PROB, SolverOpts(tile=(2, 2)), tol=1e-10)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_fmg_newton_matches_oracle(oracle_fmg, precision):
    from paper_1709_05660_gb300 import fsi
    torch.cuda.set_device(0)
    y_o, hists = oracle_fmg
    y = torch.empty(len(y_o), dtype=torch.float64, device="cuda")
    st = fsi.fmg_newton(PROB, SolverOpts(tile=(2, 2), precision=precision), y,
                        stream=torch.cuda.current_stream().cuda_stream, tol=1e-10)
    assert st["status"] == 0 and st["levels"] == 3
    for l, h in enumerate(hists):
        assert abs(st["newton_steps"][l] - len(h)) <= 1, (l, st["newton_steps"], [len(x) for x in hists])
        assert st["last_rel_step"][l] < 1e-10
    yh = y.cpu().numpy()
    assert np.linalg.norm(yh - y_o) <= 1e-8 * np.linalg.norm(y_o)


def test_fmg_rejects_transient_problems():
    from paper_1709_05660_gb300 import fsi
    y = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(fsi.FSIError) as ei:
        fsi.fmg_newton(replace(PROB, transient=1), SolverOpts(tile=(2, 2)), y)
    assert ei.value.code == -1
