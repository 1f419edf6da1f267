"""Synthetic channel-with-flap workloads and seeded inputs.

This module only describes problem data (geometry breaks, materials, solver
settings) and draws seeded random numbers.  It holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle may use it.

Geometry (stand-in for the Hron-Turek / Richter benchmark meshes, which are
not available): a rectangular channel [0,2]x[0,0.5] (x [0,0.5] in 3D) with a
Neo-Hookean flap clamped to the floor.  The coarse tensor grid is graded so
that the fluid-solid interface lies on element edges, as Sec. 2.5 requires.
Material values echo the FSI1 / FSI3 parameter tables of Sec. 4.
"""
from dataclasses import dataclass, field, replace
from typing import List, Tuple

import numpy as np


def _equal(a: float, b: float, n: int) -> List[float]:
    return [a + (b - a) * i / n for i in range(n + 1)]


def _join(*segs: List[float]) -> Tuple[float, ...]:
    out: List[float] = []
    for s in segs:
        out.extend(s if not out else s[1:])
    return tuple(out)


# Coarse cell boundaries (the x grid is 16 cells, the y grid 4 cells).
X_BREAKS = _join(_equal(0.0, 0.5, 4), _equal(0.5, 0.55, 1), _equal(0.55, 2.0, 11))
Y_BREAKS = tuple(_equal(0.0, 0.5, 4))
Z_BREAKS = (0.0, 0.1, 0.25, 0.4, 0.5)


@dataclass(frozen=True)
class Problem:
    """Problem descriptor; mirrors ``fsi_problem_desc`` of the C-ABI."""
    dim: int = 2
    breaks: Tuple[Tuple[float, ...], ...] = (X_BREAKS, Y_BREAKS)
    levels: int = 3                      # total levels, coarse level included
    flap_lo: Tuple[float, ...] = (0.5, 0.0)
    flap_hi: Tuple[float, ...] = (0.55, 0.25)
    rho_f: float = 1000.0
    mu_f: float = 1.0
    rho_s: float = 1000.0
    mu_s: float = 5e5                    # shear modulus; C1 = mu_s / 2 - mr_c2
    mr_c2: float = 0.0                   # Mooney-Rivlin C2 (0: Neo-Hookean)
    U: float = 0.2                       # mean inflow velocity
    transient: int = 0
    dt: float = 0.01
    ale_op: int = 0                      # 0: k (grad d + grad d^T), 1: k grad d


@dataclass(frozen=True)
class SolverOpts:
    """Solver options; mirrors ``fsi_solver_opts`` of the C-ABI."""
    tile: Tuple[int, ...] = (2, 2)
    n_pre: int = 2
    n_post: int = 2
    omega: float = 0.6
    restart: int = 30
    rtol: float = 1e-10
    max_iters: int = 1000
    precision: int = 0                   # 0 = FP64, 1 = mixed
    krylov: int = 0                      # 0 = FGMRES (right, true residual), 1 = GMRES (left, preconditioned residual)
    gs_passes: int = 0                   # Gram-Schmidt passes (0: 2 for FGMRES, 1 for left GMRES)
    local_solver: int = 0                # Schwarz blocks: 0 = LU for all, 1 = ILU(0) for fluid blocks, LU for solid


def problem_3d(levels: int = 3, **kw) -> Problem:
    return Problem(dim=3, breaks=(X_BREAKS, Y_BREAKS, Z_BREAKS), levels=levels,
                   flap_lo=(0.5, 0.0, 0.1), flap_hi=(0.55, 0.25, 0.4), **kw)


# The workloads: 2D channels with a flap at 3-6 levels (the 3-level one is small
# enough for the oracle to solve in seconds; the 5-level one, 313,860 unknowns,
# is the single-GPU benchmark workload) and the 3D box channel with a plate.
CONFIGS = {
    "channel2d_l3": (Problem(levels=3, mu_s=5e5, U=0.2), SolverOpts(tile=(2, 2))),
    "channel2d_l5": (Problem(levels=5, mu_s=2e6, U=1.0), SolverOpts(tile=(4, 4))),
    # the 5-level problem one level coarser (79k unknowns, ~1 GB on the device):
    # small case for detailed profiles of the same kernels
    "channel2d_l4": (Problem(levels=4, mu_s=2e6, U=1.0), SolverOpts(tile=(4, 4))),
    # 4 x 4-element Schwarz blocks (up to 372 unknowns): measured on GB300 the
    # fastest of the 4 x 4, 5 x 5 and 6 x 6 blocks (200-900 unknowns) at the
    # 1e-8 error bar - larger blocks save one or two FGMRES iterations but cost
    # n^3 to factor
    "channel2d_l6": (Problem(levels=6, mu_s=2e6, U=1.0), SolverOpts(tile=(4, 4), precision=1)),
    # 3D plate with the shear modulus of the 2D channels: softer plates (5e5)
    # deflect by more than the fluid element next to them within a few
    # steps at this inflow and tangle the mesh
    "box3d_l3_bdf2": (problem_3d(levels=3, mu_s=2e6, U=1.0, transient=1, dt=0.01),
                 SolverOpts(tile=(2, 2, 2), precision=1)),
}


def tiny_problem(levels: int = 2, **kw) -> Problem:
    """A small variant of the 2D channel used by unit tests."""
    return replace(Problem(levels=levels), **kw)


def noise(n: int, seed: int = 0, std: float = 1e-4) -> np.ndarray:
    """Seeded N(0, std^2) samples, one per unknown.

    The displacement perturbation of the benchmark state is this array
    applied at the free displacement unknowns (each side applies its own
    mask).
    """
    return np.random.default_rng(seed).standard_normal(n) * std
