"""Pins of the oracle's orthonormalisation multigrid (arXiv 2003.02431, sec. 3.3: Algorithm
ResMinimi, residual minimisation; Algorithm OrthoMG) against independent computations.

* RM: after k steps the stored W has orthonormal columns and W = M Z; x - x0 lies in the span of
  the raw directions and r = b - M x is the least-squares minimum of |r0 - M Z c| over that span
  (numpy lstsq on the raw directions, a different method than Gram-Schmidt); a direction that
  repeats an earlier one changes nothing
* OrthoMG: the residual norm never grows (the algorithm's guarantee), one two-level pass equals
  the same pass restated with dense matrices and lstsq, and the solve reaches numpy's direct
  solution; with a K-cycle (two passes per coarse visit) too
"""
import numpy as np
import pytest

import oracle
import xdg_problem as xp
from conftest import dense_from_bsr


@pytest.fixture(scope="module")
def prob():
    return xp.Problem(xp.config_2d_16(max_coarse_dof=60))


def test_rm_orthonormal_and_least_squares(prob):
    P = prob
    H = oracle.Hierarchy(P)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    rng = np.random.default_rng(1)
    b = P.b.reshape(-1)
    x0 = rng.standard_normal(P.dof) * 1e-3
    zs = rng.standard_normal((5, P.dof))
    x, r, W, Z = H.rm_steps(0, zs, b, x0)
    assert np.abs(W @ W.T - np.eye(5)).max() < 1e-12
    assert np.abs(W - (A @ Z.T).T).max() <= 1e-12 * np.abs(W).max() * np.abs(A).max() * 10
    r0 = b - A @ x0
    c, *_ = np.linalg.lstsq(A @ zs.T, r0, rcond=None)
    x_ls = x0 + zs.T @ c
    assert np.linalg.norm(x - x_ls) <= 1e-9 * np.linalg.norm(x_ls - x0)
    assert np.linalg.norm(r - (b - A @ x)) <= 1e-10 * np.linalg.norm(r0)


def test_rm_dependent_direction_changes_nothing(prob):
    P = prob
    H = oracle.Hierarchy(P)
    rng = np.random.default_rng(2)
    b = P.b.reshape(-1)
    x0 = np.zeros(P.dof)
    z1, z2 = rng.standard_normal(P.dof), rng.standard_normal(P.dof)
    xa, ra, _, _ = H.rm_steps(0, np.stack([z1, z2]), b, x0)
    xb, rb, W, Z = H.rm_steps(0, np.stack([z1, z2, 3 * z1 - 2 * z2]), b, x0)
    assert np.linalg.norm(xb - xa) <= 1e-12 * np.linalg.norm(xa)
    assert np.abs(W[2]).max() == 0.0 and np.abs(Z[2]).max() == 0.0


@pytest.mark.parametrize("passes", [1, 2])
def test_orthomg_monotone_and_reaches_dense_solution(prob, passes):
    P = prob
    oracle.set_orthomg_passes(passes)
    try:
        H = oracle.Hierarchy(P)
        A = dense_from_bsr(P.row_ptr, P.col, P.val)
        ref = np.linalg.solve(A, P.b.reshape(-1))
        x, it, rr, hist = H.orthomg(P.b, tol=1e-12, maxit=400, restart=30)
    finally:
        oracle.set_orthomg_passes(1)
    assert rr <= 1e-12 * 1.01
    assert np.all(np.diff(hist) <= 1e-15 * hist[0]), "the residual norm grew"
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_two_level_pass_matches_dense_restatement(prob):
    """One pass on a two-level hierarchy: z = D^-1 r, RM; z = R M_c^-1 R^T r, RM; z = D^-1 r, RM,
    restated with dense matrices, each RM as a least-squares fit over all directions so far."""
    P = prob
    H = oracle.Hierarchy(P, n_levels=2)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    Np = P.Np
    Dinv = np.zeros_like(A)
    for i in range(P.nb[0]):
        s = slice(i * Np, (i + 1) * Np)
        Dinv[s, s] = np.linalg.inv(A[s, s])
    Rd = np.zeros((P.dof, P.nb[1] * Np))
    for f in range(P.nb[0]):
        Rd[f * Np:(f + 1) * Np, P.agg[0][f] * Np:(P.agg[0][f] + 1) * Np] = P.R[0][f]
    b = P.b.reshape(-1)
    x0 = np.zeros(P.dof)
    r0 = b.copy()
    dirs = []

    def rm(z):
        dirs.append(z)
        Zm = np.stack(dirs, axis=1)
        c, *_ = np.linalg.lstsq(A @ Zm, r0, rcond=None)
        return x0 + Zm @ c, r0 - A @ Zm @ c

    x, r = rm(Dinv @ r0)
    x, r = rm(Rd @ np.linalg.solve(Rd.T @ A @ Rd, Rd.T @ r))
    x, r = rm(Dinv @ r)
    xo, it, rr, hist = H.orthomg(b, tol=0.0, maxit=1, restart=30)
    assert it == 1
    assert np.linalg.norm(xo - x) <= 1e-10 * np.linalg.norm(x)
    assert abs(hist[1] - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-10


def test_orthomg_restart_keeps_converging(prob):
    P = prob
    H = oracle.Hierarchy(P)
    # four passes per restart: slower than with a long memory, but still monotone and converging
    x, it, rr, hist = H.orthomg(P.b, tol=1e-11, maxit=400, restart=12)
    assert rr <= 1e-5 and np.all(np.diff(hist) <= 1e-15 * hist[0])
    _, it30, rr30, _ = H.orthomg(P.b, tol=1e-11, maxit=400, restart=30)
    assert rr30 <= 1.01e-11 and it30 < it
