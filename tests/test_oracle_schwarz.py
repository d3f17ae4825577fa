"""Pins of the oracle's additive Schwarz smoother (Algorithm Swz of arXiv 2003.02431, sec. 3.3,
with exact patch solves) against independent computations.

* dense restatement: sum_i E_i (M_{P_i P_i})^{-1} E_i^T r with numpy inverses of the dense
  patch matrices, divided by alpha (as printed: x ./ alpha) or scaled by alpha^{-1/2} on both
  sides (the symmetric form), on overlapping patches with varying alpha
* special cases: one block per patch is block Jacobi; one patch holding every block is the
  direct solve M^{-1} r; with constant alpha the printed and the symmetric forms agree
* the symmetric form is a symmetric positive definite operator; the Lanczos estimate of
  lambda_max(S M) lies within 5 % below the true value (dense eigenvalues)
* a two-level cycle with Schwarz smoothing equals the textbook formula written with dense
  matrices; the preconditioned CG reaches the dense direct solution
"""
import numpy as np
import pytest

import oracle
import xdg_problem as xp
from conftest import dense_from_bsr


@pytest.fixture(scope="module")
def prob():
    return xp.Problem(xp.config_2d_16(max_coarse_dof=60))


@pytest.fixture(scope="module")
def prob3d():
    return xp.Problem(xp.Config(D=3, N=6, k=2, c=(0.47, 0.52, 0.55), R=0.3, muA=1, muB=1000, max_coarse_dof=80))


def _staggered(P, level=1):
    a = P.schwarz_patches(level, 0)
    b = P.schwarz_patches(level, 1)
    return np.r_[a[0], a[0][-1] + b[0][1:]], np.r_[a[1], b[1]]


def _uneven(P):
    """Overlapping patches with alpha between 1 and 3: the aggregates, plus the staggered
    groups of the lower half of the blocks, plus pairs of consecutive blocks of the first tenth."""
    a = P.aggregate_patches(1)
    b = P.schwarz_patches(1, 1)
    nb = P.nb[0]
    keep = [i for i in range(len(b[0]) - 1) if b[1][b[0][i]] < nb // 2]
    ptr, blk = [0], []
    for p in range(len(a[0]) - 1):
        blk += list(a[1][a[0][p]:a[0][p + 1]])
        ptr.append(len(blk))
    for p in keep:
        blk += list(b[1][b[0][p]:b[0][p + 1]])
        ptr.append(len(blk))
    for i in range(0, nb // 10, 2):
        blk += [i, i + 1]
        ptr.append(len(blk))
    return np.array(ptr, np.int64), np.array(blk, np.int32)


def _dense_swz(A, Np, patches, mode):
    ptr, blk = patches
    n = A.shape[0]
    alpha = np.zeros(n // Np)
    for p in range(len(ptr) - 1):
        alpha[blk[ptr[p]:ptr[p + 1]]] += 1
    al = np.repeat(alpha, Np)
    S = np.zeros_like(A)
    for p in range(len(ptr) - 1):
        idx = np.concatenate([np.arange(b * Np, (b + 1) * Np) for b in blk[ptr[p]:ptr[p + 1]]])
        S[np.ix_(idx, idx)] += np.linalg.inv(A[np.ix_(idx, idx)])
    if mode == 0:
        return S / al[:, None]
    return S / np.sqrt(al)[:, None] / np.sqrt(al)[None, :]


@pytest.mark.parametrize("mode", [0, 1])
def test_schwarz_matches_dense_restatement(prob, mode):
    P = prob
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    patches = _uneven(P)
    al = np.bincount(patches[1], minlength=P.nb[0])
    assert al.min() == 1 and al.max() >= 3  # alpha really varies
    H = oracle.Hierarchy(P)
    H.set_patches(0, patches, mode=mode)
    r = np.random.default_rng(1).standard_normal(P.dof)
    ref = _dense_swz(A, P.Np, patches, mode) @ r
    z = H.schwarz(0, r)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)


def test_single_block_patches_are_block_jacobi(prob):
    P = prob
    nb, Np = P.nb[0], P.Np
    patches = (np.arange(nb + 1, dtype=np.int64), np.arange(nb, dtype=np.int32))
    H = oracle.Hierarchy(P)
    H.set_patches(0, patches)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    r = np.random.default_rng(2).standard_normal(P.dof)
    ref = np.concatenate([np.linalg.solve(A[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np], r[i * Np:(i + 1) * Np])
                          for i in range(nb)])
    assert np.linalg.norm(H.schwarz(0, r) - ref) <= 1e-11 * np.linalg.norm(ref)
    # both damping estimates (Lanczos in the M and in the D inner product, one Krylov space)
    # bound lambda_max(D^-1 M) from below within a few percent
    Dm = np.zeros_like(A)
    for i in range(nb):
        Dm[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np] = A[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np]
    lam = np.linalg.eigvals(np.linalg.solve(Dm, A)).real.max()
    for lm in (H.level(0)["lmax"], oracle.Hierarchy(P).level(0)["lmax"]):
        assert 0.95 * lam <= lm <= lam * (1 + 1e-10)


def test_one_patch_is_the_direct_solve():
    P = xp.Problem(xp.Config(D=2, N=5, k=2, c=(0.5, 0.5, 0), R=0.3, max_coarse_dof=20))
    nb = P.nb[0]
    H = oracle.Hierarchy(P)
    H.set_patches(0, (np.array([0, nb], np.int64), np.arange(nb, dtype=np.int32)))
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    r = np.random.default_rng(3).standard_normal(P.dof)
    ref = np.linalg.solve(A, r)
    assert np.linalg.norm(H.schwarz(0, r) - ref) <= 1e-10 * np.linalg.norm(ref)


def test_constant_alpha_forms_agree(prob):
    P = prob
    patches = _staggered(P)
    assert np.all(np.bincount(patches[1], minlength=P.nb[0]) == 2)  # every block in two patches
    r = np.random.default_rng(4).standard_normal(P.dof)
    out = []
    for mode in (0, 1):
        H = oracle.Hierarchy(P)
        H.set_patches(0, patches, mode=mode)
        out.append(H.schwarz(0, r))
    assert np.linalg.norm(out[0] - out[1]) <= 1e-13 * np.linalg.norm(out[1])


def test_symmetric_form_is_spd_and_lanczos_bound(prob):
    P = prob
    patches = _uneven(P)
    H = oracle.Hierarchy(P)
    H.set_patches(0, patches, mode=1)
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal(P.dof), rng.standard_normal(P.dof)
    Su, Sv = H.schwarz(0, u), H.schwarz(0, v)
    assert abs(u @ Sv - v @ Su) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(Sv)
    assert u @ Su > 0 and v @ Sv > 0
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    S = _dense_swz(A, P.Np, patches, 1)
    lam = np.linalg.eigvals(S @ A).real.max()
    lm = H.level(0)["lmax"]
    assert 0.95 * lam <= lm <= lam * (1 + 1e-10)
    assert abs(H.level(0)["omega"] - 4.0 / (3.0 * lm)) < 1e-15


def test_two_level_cycle_with_schwarz_matches_dense_formula(prob):
    P = prob
    H = oracle.Hierarchy(P, n_levels=2)
    patches = _staggered(P)
    H.set_patches(0, patches, mode=1)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    Np = P.Np
    S = _dense_swz(A, Np, patches, 1)
    Rd = np.zeros((P.dof, P.nb[1] * Np))
    for f in range(P.nb[0]):
        Rd[f * Np:(f + 1) * Np, P.agg[0][f] * Np:(P.agg[0][f] + 1) * Np] = P.R[0][f]
    om = H.level(0)["omega"]
    b = np.random.default_rng(6).standard_normal(P.dof)
    x = om * S @ b
    x = x + Rd @ np.linalg.solve(Rd.T @ A @ Rd, Rd.T @ (b - A @ x))
    x = x + om * S @ (b - A @ x)
    y = H.vcycle(b)
    assert np.linalg.norm(y - x) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_pcg_with_schwarz_matches_dense_solve(which, prob, prob3d):
    P = prob if which == "2d" else prob3d
    H = oracle.Hierarchy(P, gamma=2)
    H.set_patches(0, _staggered(P))
    if P.n_levels > 2:
        H.set_patches(1, _staggered(P, 2))
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    ref = np.linalg.solve(A, P.b.reshape(-1))
    x, it, rr, _ = H.pcg(P.b, tol=1e-13, maxit=400)
    assert rr < 1e-12
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    Hb = oracle.Hierarchy(P, gamma=2)
    assert it <= Hb.pcg(P.b, tol=1e-13, maxit=400)[1]  # overlapping Schwarz smooths at least as well


def test_invalid_patches_are_rejected(prob):
    P = prob
    H = oracle.Hierarchy(P)
    nb = P.nb[0]
    with pytest.raises(ValueError):  # block 0 in no patch
        H.set_patches(0, (np.array([0, nb - 1], np.int64), np.arange(1, nb, dtype=np.int32)))
    with pytest.raises(ValueError):  # index out of range
        H.set_patches(0, (np.array([0, 1, nb + 1], np.int64), np.r_[nb, np.arange(nb)].astype(np.int32)))
