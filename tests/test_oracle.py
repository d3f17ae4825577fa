"""Pins of the CPU oracle of the solve against independent computations.

Each oracle routine is checked against a different computation of the same mathematical
object: dense numpy products, numpy/LAPACK direct solves, direct assembly of the bilinear form
in the coarse basis (Galerkin consistency, Eq. XDGsysRestriction of arXiv 2003.02431), the
symmetry and definiteness a preconditioner for CG must have, and eigenvalue bounds.
"""
import numpy as np
import pytest

import oracle
import xdg_problem as xp
from conftest import dense_from_bsr


@pytest.fixture(scope="module")
def prob2d():
    return xp.Problem(xp.config_2d_16(max_coarse_dof=60))


@pytest.fixture(scope="module")
def prob3d():
    return xp.Problem(xp.Config(D=3, N=6, k=2, c=(0.47, 0.52, 0.55), R=0.3, muA=1, muB=1000,
                                max_coarse_dof=80))


@pytest.fixture(scope="module")
def prob3d_k5():
    """k = 5 in 3D (Np = 56, the paper's highest degree): the block size of the wide-block GPU
    kernels, three levels on 4^3 cells."""
    return xp.Problem(xp.Config(D=3, N=4, k=5, c=(0.47, 0.52, 0.55), R=0.3, muA=1, muB=1000,
                                max_coarse_dof=300))


def _prob(which, prob2d, prob3d, prob3d_k5):
    return {"2d": prob2d, "3d": prob3d, "3d_k5": prob3d_k5}[which]


def _Rdense(agg, R, nbc):
    nbf, Np = R.shape[0], R.shape[-1]
    Rd = np.zeros((nbf * Np, nbc * Np))
    for f in range(nbf):
        Rd[f * Np:(f + 1) * Np, agg[f] * Np:(agg[f] + 1) * Np] = R[f]
    return Rd


def test_spmv_matches_dense(prob2d):
    P = prob2d
    x = np.random.default_rng(1).standard_normal(P.dof)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    y = oracle.bsr_spmv(P.row_ptr, P.col, P.val, x).reshape(-1)
    assert np.abs(y - A @ x).max() <= 1e-13 * np.abs(A).max() * np.abs(x).max() * 10


def test_spmv_random_bsr():
    rng = np.random.default_rng(7)
    nb, Np = 37, 5
    rows = [sorted(rng.choice(nb, size=rng.integers(0, 6), replace=False)) for _ in range(nb)]
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    val = rng.standard_normal((len(col), Np, Np))
    x = rng.standard_normal(nb * Np)
    y = oracle.bsr_spmv(rp, col, val, x).reshape(-1)
    assert np.allclose(y, dense_from_bsr(rp, col, val) @ x, rtol=0, atol=1e-12)


@pytest.mark.parametrize("which", ["2d", "3d", "3d_k5"])
def test_transfers_match_dense(which, prob2d, prob3d, prob3d_k5):
    P = _prob(which, prob2d, prob3d, prob3d_k5)
    rng = np.random.default_rng(3)
    for l in range(P.n_levels - 1):
        Rd = _Rdense(P.agg[l], P.R[l], P.nb[l + 1])
        r = rng.standard_normal(Rd.shape[0])
        zc = rng.standard_normal(Rd.shape[1])
        x = rng.standard_normal(Rd.shape[0])
        assert np.allclose(oracle.restrict(P.agg[l], P.R[l], r, P.nb[l + 1]).reshape(-1), Rd.T @ r, atol=1e-12)
        assert np.allclose(oracle.prolong_add(P.agg[l], P.R[l], zc, x).reshape(-1), x + Rd @ zc, atol=1e-12)


@pytest.mark.parametrize("which", ["2d", "3d", "3d_k5"])
def test_galerkin_matches_dense_and_direct_assembly(which, prob2d, prob3d, prob3d_k5):
    P = _prob(which, prob2d, prob3d, prob3d_k5)
    rp, cl, vl = P.row_ptr, P.col, P.val
    for l in range(P.n_levels - 1):
        rpc, clc, vlc = oracle.galerkin(rp, cl, vl, P.agg[l], P.R[l], P.nb[l + 1])
        Rd = _Rdense(P.agg[l], P.R[l], P.nb[l + 1])
        A = dense_from_bsr(rp, cl, vl)
        Ac = dense_from_bsr(rpc, clc, vlc)
        scale = np.abs(Ac).max()
        assert np.abs(Ac - Rd.T @ A @ Rd).max() <= 1e-12 * scale
        # Galerkin consistency: a_sip assembled directly in the coarse basis. The two agree to
        # the accuracy of the orthonormal bases, built by Cholesky of Gram matrices of Legendre
        # products in graded order: ~1e-12 up to k = 3; at k = 5 the Gram matrices of small cut
        # parts are far worse conditioned (4.7e-8 measured), hence 1e-7 there.
        rpd, cld, vld, bd = P.assemble_level(l + 2)
        assert np.array_equal(rpd, rpc) and np.array_equal(cld, clc)
        assert np.abs(vld - vlc).max() <= (1e-11 if P.Np <= 20 else 1e-7) * scale
        rp, cl, vl = rpc, clc, vlc


def test_coarse_solve_matches_lapack(prob2d):
    H = oracle.Hierarchy(prob2d)
    C = H.level(H.nlev - 1)
    A = dense_from_bsr(C["row_ptr"], C["col"], C["val"])
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    z = H.coarse_solve(r)
    ref = np.linalg.solve(A, r)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)


def test_smoother_matches_dense(prob2d):
    H = oracle.Hierarchy(prob2d)
    P = prob2d
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    Np = P.Np
    Dm = np.zeros_like(A)
    for i in range(P.nb[0]):
        Dm[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np] = A[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np]
    rng = np.random.default_rng(9)
    b, x = rng.standard_normal(P.dof), rng.standard_normal(P.dof)
    om = H.level(0)["omega"]
    ref = x + om * np.linalg.solve(Dm, b - A @ x)
    y = H.smooth(0, b, x)
    assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max()
    # Lanczos estimate: a lower bound of lambda_max(D^-1 A) within a few percent
    lam = np.linalg.eigvals(np.linalg.solve(Dm, A)).real.max()
    lm = H.level(0)["lmax"]
    assert lm <= lam * (1 + 1e-10) and lm >= 0.95 * lam
    assert abs(om - 4.0 / (3.0 * lm)) < 1e-15


def test_k5_smoother_spmv_and_solve_match_dense(prob3d_k5):
    """Np = 56: the operator apply, one damped block-Jacobi step and the PCG solution against
    dense numpy / LAPACK."""
    P = prob3d_k5
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    rng = np.random.default_rng(13)
    x = rng.standard_normal(P.dof)
    y = oracle.bsr_spmv(P.row_ptr, P.col, P.val, x).reshape(-1)
    assert np.abs(y - A @ x).max() <= 1e-12 * np.abs(A).max() * np.abs(x).max() * 10
    H = oracle.Hierarchy(P)
    Np = P.Np
    Dm = np.zeros_like(A)
    for i in range(P.nb[0]):
        Dm[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np] = A[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np]
    b = rng.standard_normal(P.dof)
    om = H.level(0)["omega"]
    ref = x + om * np.linalg.solve(Dm, b - A @ x)
    assert np.abs(H.smooth(0, b, x) - ref).max() <= 1e-10 * np.abs(ref).max()
    sol, it, rr, _ = H.pcg(P.b, tol=1e-13, maxit=600)
    dense = np.linalg.solve(A, P.b.reshape(-1))
    assert rr <= 1e-13 and np.linalg.norm(sol - dense) <= 1e-8 * np.linalg.norm(dense), it


@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_symmetric_positive(prob3d, gamma):
    H = oracle.Hierarchy(prob3d, gamma=gamma)
    rng = np.random.default_rng(11)
    u, v = rng.standard_normal(H.n), rng.standard_normal(H.n)
    Bu, Bv = H.vcycle(u), H.vcycle(v)
    assert abs(u @ Bv - v @ Bu) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(Bv)
    assert u @ Bu > 0 and v @ Bv > 0


def test_cycle_single_level_is_direct_solve(prob2d):
    P = xp.Problem(xp.Config(D=2, N=6, k=2, c=(0.5, 0.5, 0), R=0.3, max_levels=1))
    H = oracle.Hierarchy(P)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    b = P.b.reshape(-1)
    assert np.linalg.norm(H.vcycle(b) - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(np.linalg.solve(A, b))


def test_two_level_cycle_matches_dense_formula(prob2d):
    # V(1,1) with an exact coarse solve written as dense matrices
    P = prob2d
    H = oracle.Hierarchy(P, n_levels=2)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    Np = P.Np
    Dm = np.zeros_like(A)
    for i in range(P.nb[0]):
        Dm[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np] = A[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np]
    Rd = _Rdense(P.agg[0], P.R[0], P.nb[1])
    om = H.level(0)["omega"]
    b = np.random.default_rng(2).standard_normal(P.dof)
    x = om * np.linalg.solve(Dm, b)
    x = x + Rd @ np.linalg.solve(Rd.T @ A @ Rd, Rd.T @ (b - A @ x))
    x = x + om * np.linalg.solve(Dm, b - A @ x)
    y = H.vcycle(b)
    assert np.linalg.norm(y - x) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_pcg_matches_dense_solve(which, prob2d, prob3d):
    P = prob2d if which == "2d" else prob3d
    H = oracle.Hierarchy(P, gamma=2)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    ref = np.linalg.solve(A, P.b.reshape(-1))
    x, it, rr, hist = H.pcg(P.b, tol=1e-13, maxit=400)
    assert rr < 1e-12
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_mesh_independent_iterations_2d():
    # iteration counts of the multigrid-preconditioned CG stay nearly constant under refinement
    its = []
    for N in (32, 64, 128):
        P = xp.Problem(xp.Config(D=2, N=N, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000, max_coarse_dof=300))
        H = oracle.Hierarchy(P, gamma=2)
        its.append(H.pcg(P.b, tol=1e-10, maxit=400)[1])
    assert max(its) <= 1.25 * min(its), its


def test_mesh_independent_iterations_3d():
    # sec. 4: the iteration counts of the multigrid solvers stay nearly independent of the mesh.
    # The 3D workload (sphere R = 0.31, mu 1:1000, k = 2, W-cycle on the two finest levels) at
    # N = 16, 24, 32: the counts move with how the sphere cuts each mesh (56, 48, 56), so the
    # pin is a bounded spread and no growth from the coarsest to the finest mesh, not +-2.
    its = []
    for N in (16, 24, 32):
        P = xp.Problem(xp.config_3d_64(N=N, max_coarse_dof=1000))
        H = oracle.Hierarchy(P, gamma=2)
        oracle.set_w_levels(H, 2)
        its.append(H.pcg(P.b, tol=1e-10, maxit=400)[1])
    assert max(its) <= 1.2 * min(its), its
    assert its[-1] <= its[0] + 2, its


def test_quantized_storage_rounding():
    # FP32 storage: entry/scale rounded to float; BF16: further rounded to bfloat16 with ties to
    # even -- checked against torch's float32 -> bfloat16 conversion
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    a = rng.standard_normal((200, 6, 6)) * np.exp(rng.uniform(-20, 20, (200, 1, 1)))
    a[3] = 0.0
    for prec in (1, 2):
        q, s = oracle.quantize_blocks(a, prec)
        m = np.abs(a).reshape(200, -1).max(axis=1)
        assert np.array_equal(s, np.where(m > 0, m, 1.0).astype(np.float32))
        ratio = (a.reshape(200, -1) / s.astype(np.float64)[:, None]).astype(np.float32)
        if prec == 2:
            ratio = torch.from_numpy(ratio).to(torch.bfloat16).to(torch.float32).numpy()
        expect = s.astype(np.float64)[:, None] * ratio.astype(np.float64)
        assert np.array_equal(q.reshape(200, -1), expect)
        assert np.all(q[3] == 0.0)


def _blockdiag(A, Np):
    D = np.zeros_like(A)
    for i in range(A.shape[0] // Np):
        D[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np] = A[i * Np:(i + 1) * Np, i * Np:(i + 1) * Np]
    return D


@pytest.mark.parametrize("wlev", [0, 1, 2])
def test_w_cycle_matches_dense_recursion(wlev):
    """The W-cycle (gamma = 2) and its restriction to the wlev finest levels (V below), written
    as the textbook recursion with dense matrices: pre-smoothing from zero, restriction, gamma
    coarse steps z_c += B_c(r_c - M_c z_c) on levels l < wlev (one step below), prolongation,
    post-smoothing; Galerkin coarse matrices; exact coarsest solve. Four levels."""
    P = xp.Problem(xp.Config(D=2, N=16, k=2, c=(0.5, 0.5, 0), R=0.3, muA=1, muB=10, max_coarse_dof=20,
                                max_levels=4))
    assert P.n_levels == 4
    H = oracle.Hierarchy(P, gamma=2)
    if wlev:
        oracle.set_w_levels(H, wlev)
    Np, nl = P.Np, P.n_levels
    A = [dense_from_bsr(P.row_ptr, P.col, P.val)]
    Rd = []
    for l in range(nl - 1):
        Rd.append(_Rdense(P.agg[l], P.R[l], P.nb[l + 1]))
        A.append(Rd[l].T @ A[l] @ Rd[l])
    om = [H.level(l)["omega"] for l in range(nl - 1)]
    wl = wlev if wlev else nl

    def B(l, b):
        if l == nl - 1:
            return np.linalg.solve(A[l], b)
        D = _blockdiag(A[l], Np)
        x = om[l] * np.linalg.solve(D, b)
        bc = Rd[l].T @ (b - A[l] @ x)
        zc = B(l + 1, bc)
        if l + 2 < nl and l < wl:
            zc = zc + B(l + 1, bc - A[l + 1] @ zc)
        x = x + Rd[l] @ zc
        return x + om[l] * np.linalg.solve(D, b - A[l] @ x)

    b = np.random.default_rng(21).standard_normal(P.dof)
    ref = B(0, b)
    got = H.vcycle(b)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref), wlev
    H.close()
