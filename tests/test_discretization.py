"""Pins of the XDG-SIP system generator against what the paper and the mathematics fix.

Kummer, Smuda, Weber, arXiv 2003.02431:
  * cut-cell quadrature (sec. 2.1, Saye's method): closed-form volumes and interface areas
  * DOF table of the performance study (Table tab:DOFs, sec. 4): exact integers
  * SIP operator (Eq. DefSIP): symmetric positive definite (the paper calls the system SPD, sec. 4)
  * consistency: a solution inside the discrete space is reproduced exactly (patch test)
  * h^{k+1} convergence under refinement (sec. 5)
  * orthonormal level bases, so (R^{X,lambda})^T restricted to one aggregate is an L2 projector
    (sec. 3.2): sum_f R_f^T R_f = I per coarse block
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import oracle
import xdg_problem as xp
from conftest import dense_from_bsr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dof_table.txt")


def _sparse(P):
    nb, Np = P.nb[0], P.Np
    return sp.bsr_matrix((P.val, P.col, P.row_ptr), shape=(nb * Np, nb * Np)).tocsc()


# ------------------------------------------------------------------ quadrature closed forms
@pytest.mark.parametrize("c,N", [((0.5, 0.5), 16), ((0.5, 0.5), 5), ((0.437, 0.561), 12), ((0.5, 0.3), 8)])
def test_circle_area_and_perimeter(c, N):
    R = 0.27
    P = xp.Problem(xp.Config(D=2, N=N, k=2, c=(c[0], c[1], 0.0), R=R, max_levels=1))
    assert abs(P.info["volA"] - math.pi * R * R) < 1e-13
    assert abs(P.info["areaI"] - 2 * math.pi * R) < 1e-12
    assert abs(P.info["volA"] + P.info["volB"] - 1.0) < 1e-13


@pytest.mark.parametrize("c,N,R", [((0.5, 0.5, 0.5), 4, 0.3), ((0.47, 0.52, 0.55), 6, 0.3),
                                   ((0.5, 0.5, 0.5), 16, 0.31), ((0.5, 0.5, 0.5), 2, 0.3),
                                   ((0.5001, 0.4999, 0.5), 4, 0.26)])
def test_sphere_volume_and_area(c, N, R):
    # includes a centre on a grid vertex with h < R < h*sqrt(3) (square-root branches at
    # cell faces) and a centre 1e-4 away from a vertex (near-branches)
    P = xp.Problem(xp.Config(D=3, N=N, k=2, c=c, R=R, max_levels=1))
    V, A = 4.0 / 3.0 * math.pi * R ** 3, 4 * math.pi * R * R
    assert abs(P.info["volA"] / V - 1) < 1e-11
    assert abs(P.info["areaI"] / A - 1) < 1e-10
    assert abs(P.info["volA"] + P.info["volB"] - 1.0) < 1e-13


# ------------------------------------------------------------------ DOF table (hard integer pin)
def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, N, dof = map(int, line.split())
            rows.append((k, N, dof))
    return rows


@pytest.mark.parametrize("k,N,dof", [r for r in _golden() if r[0] == 2])
def test_dof_table_k2(k, N, dof):
    P = xp.Problem(xp.config_paper_twin(N, k, max_levels=1))
    assert P.dof == dof


@pytest.mark.parametrize("k,N,dof", [r for r in _golden() if r[0] != 2 and r[1] <= 8])
def test_dof_table_k3_k5_small(k, N, dof):
    # the block count does not depend on k; the k=3 and k=5 rows follow with Np = 20, 56
    P = xp.Problem(xp.config_paper_twin(N, k, max_levels=1))
    assert P.dof == dof


def test_dof_table_blocks_for_all_degrees():
    rows = _golden()
    blocks = {N: dof // math.comb(2 + 3, 3) for k, N, dof in rows if k == 2}
    for k, N, dof in rows:
        assert dof == blocks[N] * math.comb(k + 3, 3)


# ------------------------------------------------------------------ operator properties
@pytest.mark.parametrize("k", [4, 5])
def test_symmetric_positive_definite_high_degree_3d(k):
    """The 3D k = 4 and k = 5 operators (Np = 35, 56; the blocks of the wide-block GPU
    kernels) are exactly symmetric and positive definite (one cut configuration each)."""
    P = xp.Problem(xp.Config(D=3, N=3, k=k, c=(0.5, 0.47, 0.52), R=0.3, muA=1, muB=1000, max_levels=1))
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A)[0] > 0


@pytest.mark.parametrize("D,N,k", [(2, 6, 2), (2, 6, 3), (2, 5, 4), (3, 3, 2), (3, 3, 3)])
def test_symmetric_positive_definite(D, N, k):
    rng = np.random.default_rng(D * 100 + N * 10 + k)
    for _ in range(3):
        c = tuple(rng.uniform(0.35, 0.65, 3))
        R = rng.uniform(0.15, 0.4)
        P = xp.Problem(xp.Config(D=D, N=N, k=k, c=c, R=R, muA=1, muB=1000, max_levels=1))
        A = dense_from_bsr(P.row_ptr, P.col, P.val)
        assert np.array_equal(A, A.T)
        assert np.linalg.eigvalsh(0.5 * (A + A.T))[0] > 0


@pytest.mark.parametrize("D,N,k,c,mu", [(2, 8, 2, (0.5, 0.5, 0), 10.0), (2, 7, 3, (0.51, 0.47, 0), 1000.0),
                                        (3, 4, 2, (0.5, 0.5, 0.5), 10.0), (3, 5, 2, (0.47, 0.52, 0.55), 1000.0),
                                        (3, 3, 3, (0.45, 0.5, 0.52), 100.0)])
def test_patch_quadratic_solution_reproduced(D, N, k, c, mu):
    # u_s = phi/mu_s has [u] = 0 and [mu grad u . n] = 0 on the interface and -mu_s Lap u_s = -2D
    # in both species; it lies in the agglomerated space for k >= 2, so SIP reproduces it.
    P = xp.Problem(xp.Config(D=D, N=N, k=k, c=c, R=0.3, muA=1, muB=mu, rhs_kind=1, max_levels=1))
    x = spl.spsolve(_sparse(P), P.b.reshape(-1))
    e, n = P.l2_error(x)
    assert e / n < 1e-10


def _rate(D, k, Ns, mu=10.0):
    # discrete solutions from the oracle's multigrid-preconditioned CG (itself pinned against
    # dense direct solves in test_oracle.py), converged far below the discretisation error
    errs = []
    for N in Ns:
        P = xp.Problem(xp.Config(D=D, N=N, k=k, c=(0.5, 0.5, 0.5), R=0.3, muA=1, muB=mu, max_coarse_dof=400))
        x, it, rr, _ = oracle.Hierarchy(P, gamma=2).pcg(P.b, tol=1e-13, maxit=500)
        assert rr < 1e-12
        errs.append(P.l2_error(x)[0])
    return [math.log(errs[i] / errs[i + 1]) / math.log(Ns[i + 1] / Ns[i]) for i in range(len(Ns) - 1)]


def test_convergence_rate_2d_k2():
    assert min(_rate(2, 2, [16, 32, 64])) > 2.8


def test_convergence_rate_2d_k3():
    assert min(_rate(2, 3, [8, 16, 32])) > 3.7


def test_convergence_rate_3d_k2():
    assert min(_rate(3, 2, [12, 16, 24])) > 2.7


# ------------------------------------------------------------------ level bases and transfers
@pytest.mark.parametrize("cfg", [xp.config_2d_16(max_coarse_dof=50),
                                 xp.Config(D=3, N=8, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000,
                                           max_coarse_dof=50)])
def test_transfer_is_orthonormal_projection(cfg):
    P = xp.Problem(cfg)
    assert P.n_levels >= 3
    Np = P.Np
    for l in range(P.n_levels - 1):
        nbc = P.nb[l + 1]
        S = np.zeros((nbc, Np, Np))
        np.add.at(S, P.agg[l], np.einsum("fmi,fmj->fij", P.R[l], P.R[l]))
        assert np.abs(S - np.eye(Np)).max() < 1e-11


def test_levels_nested_and_ordered():
    P = xp.Problem(xp.Config(D=3, N=8, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000, max_coarse_dof=50))
    for l in range(P.n_levels):
        m = P.level_meta(l + 1)
        key = m["rep"].astype(np.int64) * 2 + m["species"]
        assert np.all(np.diff(key) > 0)  # (representative cell, species) strictly increasing
    for l in range(P.n_levels - 1):
        a = P.agg[l]
        assert a.min() >= 0 and a.max() == P.nb[l + 1] - 1
        assert len(np.unique(a)) == P.nb[l + 1]  # every coarse block has a child
        mf, mc = P.level_meta(l + 1), P.level_meta(l + 2)
        assert np.all(mf["species"] == mc["species"][a])  # no aggregation across the interface
        assert np.all(mc["rep"][a] <= mf["rep"])
