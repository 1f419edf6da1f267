"""Pins of the oracle's V-cycle (Sec. 3, 3.3) against closed forms (CPU only).

A V-cycle applied to b from x = 0 is a linear stationary method, so its
output is (I - E) J^{-1} b with E its error-propagation operator.  For two
levels with exact coarse solves, E = K_s^{n_post} K_c K_s^{n_pre}, where
K_s = I - omega S J is the Richardson step with the restricted additive
Schwarz operator S = sum_k (R^0_k)^T B_k^{-1} R^delta_k and K_c =
I - P A_0^{-1} R J the coarse-grid correction.  The tests build E from dense
matrices (numpy inverses, independent of the oracle's sequencing of
smoothing, residuals, restriction, recursion and prolongation) and compare:

* no smoothing: the cycle is the coarse-grid correction P A_0^{-1} R b;
* one subdomain covering the fine level, omega = 1: one pre-smoothing step
  is an exact solve, so the cycle returns J^{-1} b;
* 2 + 2 steps with omega = 0.6 on 2 x 2-element blocks: the full product.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import solver
from oracle.mesh import Patch, initial_state
from paper_1709_05660_gb300.workloads import Problem, SolverOpts, noise

# 4 x 2 coarse cells with the flap on element edges; two levels (8 x 4 fine)
PROB = Problem(breaks=((0.0, 0.5, 0.55, 1.0, 2.0), (0.0, 0.25, 0.5)), levels=2, mu_s=5e5, U=0.2)


def _oracle(opts):
    orc = solver.Oracle(PROB, opts)
    y = initial_state(PROB, orc.fine, noise(orc.fine.N, 0))
    orc.assemble(y)
    return orc


def _schwarz_dense(ops):
    n = ops.J.shape[0]
    Jd = ops.J.toarray()
    S = np.zeros((n, n))
    for pt in ops.patches:
        idx = np.asarray(pt.dofs)
        Binv = np.linalg.inv(Jd[np.ix_(idx, idx)])
        own = idx[np.asarray(pt.owned, dtype=bool)]
        S[own[:, None], idx[None, :]] += Binv[np.asarray(pt.owned, dtype=bool)]
    return S


def _two_grid_dense(orc, opts):
    """(I - E) J^{-1} as a dense matrix for the two-level cycle of `opts`."""
    f, c = orc.ops[1], orc.ops[0]
    J = f.J.toarray()
    n = J.shape[0]
    P, R = f.P.toarray(), f.R.toarray()
    Kc = np.eye(n) - P @ np.linalg.solve(c.J.toarray(), R @ J)
    Ks = np.eye(n) - opts.omega * _schwarz_dense(f) @ J
    E = np.linalg.matrix_power(Ks, opts.n_post) @ Kc @ np.linalg.matrix_power(Ks, opts.n_pre)
    return (np.eye(n) - E) @ np.linalg.inv(J)


def _rhs(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


def test_vcycle_without_smoothing_is_the_coarse_correction():
    opts = SolverOpts(tile=(2, 2), n_pre=0, n_post=0)
    orc = _oracle(opts)
    orc.factor()
    f, c = orc.ops[1], orc.ops[0]
    b = _rhs(f.J.shape[0], 1)
    want = f.P @ np.linalg.solve(c.J.toarray(), f.R @ b)
    got = orc.precond(b)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_vcycle_with_an_exact_smoother_is_a_direct_solve():
    opts = SolverOpts(tile=(2, 2), n_pre=1, n_post=1, omega=1.0)
    orc = _oracle(opts)
    lev = orc.fine
    whole = Patch(elems=np.arange(lev.n_elem), dofs=np.arange(lev.N), owned=np.ones(lev.N, dtype=bool), solid=False)
    orc.ops[1].patches = [whole]
    orc.factor()
    b = _rhs(lev.N, 2)
    want = np.linalg.solve(orc.ops[1].J.toarray(), b)
    got = orc.precond(b)
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)


@pytest.mark.parametrize("n_pre,n_post,omega", [(2, 2, 0.6), (1, 3, 0.7), (0, 1, 0.6)])
def test_vcycle_equals_its_error_propagation_form(n_pre, n_post, omega):
    opts = SolverOpts(tile=(2, 2), n_pre=n_pre, n_post=n_post, omega=omega)
    orc = _oracle(opts)
    orc.factor()
    assert len(orc.ops[1].patches) >= 4
    M = _two_grid_dense(orc, opts)
    for seed in (3, 4):
        b = _rhs(M.shape[0], seed)
        want = M @ b
        got = orc.precond(b)
        assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want), (n_pre, n_post, omega)


def test_vcycle_is_linear_in_the_right_hand_side():
    opts = SolverOpts(tile=(2, 2))
    orc = _oracle(opts)
    orc.factor()
    n = orc.fine.N
    b1, b2 = _rhs(n, 5), _rhs(n, 6)
    lhs = orc.precond(2.0 * b1 - 3.0 * b2)
    rhs = 2.0 * orc.precond(b1) - 3.0 * orc.precond(b2)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)
