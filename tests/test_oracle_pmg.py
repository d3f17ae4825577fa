"""Pins of the oracle's p-multigrid (arXiv 2003.02431, sec. 3.3, Algorithm pMultigrid).

* dense restatement: the low-order system M[I_lo, I_lo] solved with numpy, the residual, then
  every block's high-order system solved with numpy on the residual, on all blocks and on a
  block subset I (the Schwarz-block use of the algorithm)
* special cases: no low-order modes is block Jacobi, every mode low-order is the direct solve
* the low-order modes of the graded basis span the polynomials up to degree k_lo: for the
  patch-test solution u = phi / mu (quadratic, reproduced exactly by k >= 2), the k_lo = 2 low
  system alone already solves the problem
"""
import numpy as np
import pytest

import oracle
import xdg_problem as xp
from conftest import dense_from_bsr


@pytest.fixture(scope="module")
def prob():
    return xp.Problem(xp.Config(D=2, N=12, k=3, c=(0.5, 0.5, 0), R=0.3, muA=1, muB=100, max_coarse_dof=100))


def _dense_pmg(A, Np, n_lo, b, blocks):
    x = np.zeros_like(b)
    lo = np.concatenate([np.arange(i * Np, i * Np + n_lo) for i in blocks])
    if len(lo):
        x[lo] = np.linalg.solve(A[np.ix_(lo, lo)], b[lo])
    r = b - A @ x
    for j in blocks:
        hi = np.arange(j * Np + n_lo, (j + 1) * Np)
        if len(hi):
            x[hi] += np.linalg.solve(A[np.ix_(hi, hi)], r[hi])
    return x


@pytest.mark.parametrize("n_lo", [1, 3, 6])
def test_pmg_matches_dense_restatement(prob, n_lo):
    P = prob
    H = oracle.Hierarchy(P)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    b = np.random.default_rng(1).standard_normal(P.dof)
    ref = _dense_pmg(A, P.Np, n_lo, b, range(P.nb[0]))
    assert np.linalg.norm(H.pmg(0, n_lo, b) - ref) <= 1e-10 * np.linalg.norm(ref)
    sub = np.arange(0, P.nb[0], 3, dtype=np.int32)
    ref_sub = _dense_pmg(A, P.Np, n_lo, b, sub)
    got = H.pmg(0, n_lo, b, sub)
    assert np.linalg.norm(got - ref_sub) <= 1e-10 * np.linalg.norm(ref_sub)
    out = np.setdiff1d(np.arange(P.nb[0]), sub)
    assert np.all(got.reshape(-1, P.Np)[out] == 0.0)


@pytest.fixture(scope="module")
def prob_k5():
    return xp.Problem(xp.Config(D=3, N=3, k=5, c=(0.5, 0.47, 0.52), R=0.3, muA=1, muB=1000, max_levels=2))


@pytest.mark.parametrize("n_lo", [4, 20])
def test_pmg_k5_matches_dense_restatement(prob_k5, n_lo):
    """3D k = 5 (Np = 56) with the paper's low orders k_lo = 1 and 3 (n_lo = 4, 20): the
    reference of the GPU's wide-block p-multigrid tests."""
    P = prob_k5
    H = oracle.Hierarchy(P)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    b = np.random.default_rng(3).standard_normal(P.dof)
    ref = _dense_pmg(A, P.Np, n_lo, b, range(P.nb[0]))
    assert np.linalg.norm(H.pmg(0, n_lo, b) - ref) <= 1e-10 * np.linalg.norm(ref)


def test_pmg_special_cases(prob):
    P = prob
    H = oracle.Hierarchy(P)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    b = np.random.default_rng(2).standard_normal(P.dof)
    Np = P.Np
    bj = np.concatenate([np.linalg.solve(A[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np], b[i * Np:(i + 1) * Np])
                         for i in range(P.nb[0])])
    assert np.linalg.norm(H.pmg(0, 0, b) - bj) <= 1e-11 * np.linalg.norm(bj)
    direct = np.linalg.solve(A, b)
    assert np.linalg.norm(H.pmg(0, Np, b) - direct) <= 1e-10 * np.linalg.norm(direct)


def test_low_order_modes_span_the_low_degree_polynomials():
    # quadratic manufactured solution u_s = phi / mu_s, exactly representable for k >= 2
    P = xp.Problem(xp.Config(D=2, N=10, k=3, c=(0.5, 0.5, 0), R=0.3, muA=1, muB=10, rhs_kind=1,
                             max_coarse_dof=100))
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    exact = np.linalg.solve(A, P.b.reshape(-1))
    Np, n_lo = P.Np, 6  # k_lo = 2 in 2D
    hi = exact.reshape(-1, Np)[:, n_lo:]
    assert np.abs(hi).max() <= 1e-9 * np.abs(exact).max()  # the solution lies in the low modes
    H = oracle.Hierarchy(P)
    x = H.pmg(0, n_lo, P.b.reshape(-1))
    assert np.linalg.norm(x - exact) <= 1e-8 * np.linalg.norm(exact)
