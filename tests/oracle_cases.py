"""Small problem definitions shared by the oracle pin tests (test data only)."""
from dataclasses import replace

import numpy as np

from paper_1709_05660_gb300.workloads import Problem, SolverOpts, X_BREAKS, Y_BREAKS

# 2D channel, coarse 16x4 graded grid (interface on element edges)
CHANNEL_2D = Problem(levels=2, mu_s=5e5, U=0.2)

# small 3D channel: 3x2x3 coarse hexahedra, one of them solid
SMALL_3D = Problem(dim=3, breaks=((0.0, 0.5, 0.55, 1.0), (0.0, 0.25, 0.5), (0.0, 0.1, 0.4, 0.5)),
                   levels=1, flap_lo=(0.5, 0.0, 0.1), flap_hi=(0.55, 0.25, 0.4),
                   mu_s=5e5, U=0.5)

# unit square, 2x2 coarse cells; flap box outside (all fluid) or covering it
UNIT_FLUID = Problem(breaks=((0.0, 0.5, 1.0), (0.0, 0.5, 1.0)), levels=1,
                     flap_lo=(5.0, 5.0), flap_hi=(6.0, 6.0), rho_f=1.0, mu_f=1.0, U=0.0)
UNIT_SOLID = Problem(breaks=((0.0, 0.5, 1.0), (0.0, 0.5, 1.0)), levels=1,
                     flap_lo=(-1.0, -1.0), flap_hi=(2.0, 2.0), rho_s=1.0, mu_s=1.0, U=0.0)


def random_state(lev, seed=0, d_amp=1e-3, u_amp=0.3, p_amp=50.0):
    """A generic state exercising every term: nonzero d, u and p."""
    rng = np.random.default_rng(seed)
    y = np.zeros(lev.N)
    nd = 2 * lev.dim
    nn = lev.n_nodes * nd
    for c in range(lev.dim):
        y[c:nn:nd] = d_amp * rng.standard_normal(lev.n_nodes)
        y[lev.dim + c:nn:nd] = u_amp * rng.standard_normal(lev.n_nodes)
    y[nn:] = p_amp * rng.standard_normal(lev.N - nn)
    return y
