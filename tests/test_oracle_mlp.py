"""Pins of the learned-correction oracle (oracle/mlp.py) against what mathematics fixes:

* GELU = x Phi(x) at points where the normal distribution function is tabulated
* its derivative and the network gradient against central finite differences (FP64)
* the loss at closed-form points: exact local solve -> -1, zero -> 0, twice the local solve -> 0
* the energy identity behind the loss: for a correction on one unit, the change of the
  M-norm of the true error (from a dense direct solve) equals delta^T M_uu delta - 2 delta^T r_u
* unit matrices equal the dense operator's submatrices; units pair an A block with a B block
"""
import numpy as np
import pytest

import xdg_problem as xp
from conftest import dense_from_bsr
from oracle import mlp


def test_gelu_tabulated_values():
    # Phi(0) = 1/2, Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208 (normal tables)
    x = np.array([0.0, 1.0, -1.0, 2.0, -2.0])
    ref = np.array([0.0, 0.8413447460685429, -(1 - 0.8413447460685429), 2 * 0.9772498680518208,
                    -2 * (1 - 0.9772498680518208)])
    assert np.allclose(mlp.gelu(x), ref, rtol=0, atol=1e-15)


def test_gelu_grad_finite_difference():
    x = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(x)).max() < 1e-9


def _random_case(rng, S=7, n_in=9, n_out=6):
    lay, total = mlp.layout(n_in, n_out)
    theta = rng.standard_normal(total) * 0.3
    X = rng.standard_normal((S, n_in))
    A = rng.standard_normal((S, n_out, n_out))
    M = np.einsum("sij,skj->sik", A, A) + n_out * np.eye(n_out)
    R = rng.standard_normal((S, n_out))
    c = mlp.optimal_decrease(M, R)
    return theta, X, M, R, c


def test_loss_closed_form_points():
    rng = np.random.default_rng(0)
    _, _, M, R, c = _random_case(rng)
    ystar = np.linalg.solve(M, R[..., None])[..., 0]
    L, _ = mlp.loss(ystar, M, R, c)
    assert np.allclose(L, -1.0, atol=1e-12)
    L0, _ = mlp.loss(np.zeros_like(R), M, R, c)
    assert np.allclose(L0, 0.0)
    L2, _ = mlp.loss(2 * ystar, M, R, c)
    assert np.allclose(L2, 0.0, atol=1e-12)


def test_loss_gradient_in_y_finite_difference():
    rng = np.random.default_rng(1)
    _, _, M, R, c = _random_case(rng)
    Y = rng.standard_normal(R.shape)
    L, dY = mlp.loss(Y, M, R, c)
    h = 1e-6
    for s in range(Y.shape[0]):
        for j in range(Y.shape[1]):
            E = np.zeros_like(Y)
            E[s, j] = h
            fd = (mlp.loss(Y + E, M, R, c)[0][s] - mlp.loss(Y - E, M, R, c)[0][s]) / (2 * h)
            assert abs(fd - dY[s, j]) < 1e-6 * max(1.0, abs(dY[s, j]))


def test_parameter_gradient_finite_difference():
    rng = np.random.default_rng(2)
    theta, X, M, R, c = _random_case(rng)
    L, g = mlp.mean_loss_and_grad(theta, X, M, R, c)
    h = 1e-4
    # central differences: truncation of order h^2, rounding of order 1e-16 |L| / h
    slack = 1e-15 * abs(L) / h

    def fd(d):
        return (mlp.mean_loss_and_grad(theta + h * d, X, M, R, c)[0]
                - mlp.mean_loss_and_grad(theta - h * d, X, M, R, c)[0]) / (2 * h)

    idx = np.concatenate([np.arange(0, 20), rng.choice(theta.size, 200, replace=False), [theta.size - 1]])
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = 1.0
        assert abs(fd(e) - g[i]) < 1e-6 * max(1.0, abs(g[i])) + slack, i
    # directional derivatives along random directions
    for _ in range(3):
        d = rng.standard_normal(theta.size)
        assert abs(fd(d) - g @ d) < 1e-5 * max(1.0, abs(g @ d)) + 10 * slack


@pytest.fixture(scope="module")
def small_problem():
    P = xp.Problem(xp.Config(D=2, N=10, k=2, c=(0.47, 0.52, 0), R=0.27, muA=1, muB=50, max_coarse_dof=60))
    return P


def test_units_pair_species_blocks(small_problem):
    P = small_problem
    pairs, geom, cells = P.learned_units()
    opairs, ocells = mlp.unit_pairs(P.cut_cells())
    assert np.array_equal(pairs, opairs) and np.array_equal(cells, ocells)
    sp = P.level_meta(1)["species"]
    assert np.all(sp[pairs[:, 0]] == 0) and np.all(sp[pairs[:, 1]] == 1)
    assert len({tuple(p) for p in pairs}) == len(pairs)
    # every cut cell's blocks are a unit
    assert {tuple(x) for x in P.cut_cells()[:, 1:]} == {tuple(p) for p in pairs}
    assert geom.shape == (len(pairs), 4 + 3)


def test_unit_matrices_are_submatrices(small_problem):
    P = small_problem
    pairs, _, _ = P.learned_units()
    Mu = mlp.unit_matrices(P.row_ptr, P.col, P.val, pairs)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    Np = P.Np
    for u, (a, b) in enumerate(pairs):
        ii = np.r_[a * Np:(a + 1) * Np, b * Np:(b + 1) * Np]
        assert np.array_equal(Mu[u], A[np.ix_(ii, ii)])


def test_energy_identity_and_learned_step(small_problem):
    """The accepted corrections lower the true error's energy by exactly -E for one unit."""
    P = small_problem
    Np = P.Np
    pairs, geom, _ = P.learned_units()
    Mu = mlp.unit_matrices(P.row_ptr, P.col, P.val, pairs)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    b = P.b.reshape(-1)
    xstar = np.linalg.solve(A, b)
    rng = np.random.default_rng(3)
    z = xstar + 0.1 * rng.standard_normal(xstar.size)
    r = b - A @ z
    n_in, n_out = geom.shape[1] + 2 * Np, 2 * Np
    _, total = mlp.layout(n_in, n_out)
    theta = rng.standard_normal(total) * 0.05
    # one unit at a time: energy change from the dense solution vs the local formula
    for u in range(min(5, len(pairs))):
        sel = np.array([u])
        z1, keep, E = mlp.learned_step(theta, geom[sel], pairs[sel], Mu[sel], r, z, n_out, 1.0)
        e0, e1 = xstar - z, xstar - z1
        dE = e1 @ A @ e1 - e0 @ A @ e0
        if keep[0]:
            assert dE < 0
            assert abs(dE - E[0]) < 1e-9 * max(1.0, abs(E[0]))
        else:
            assert np.array_equal(z1, z)
    # the exact local solve in block-Jacobi coordinates: energy change -c s^2, and
    # delta = s Xu^T y* equals M_uu^{-1} r_u
    Xu, H = mlp.unit_transform(Mu)
    X, rhat, s = mlp.unit_inputs(geom, pairs, r, Xu)
    ystar = np.linalg.solve(H, rhat[..., None])[..., 0]
    delta = np.einsum("uji,uj->ui", Xu, ystar) * s[:, None]
    ru = np.concatenate([r.reshape(-1, Np)[pairs[:, 0]], r.reshape(-1, Np)[pairs[:, 1]]], axis=1)
    assert np.allclose(delta, np.linalg.solve(Mu, ru[..., None])[..., 0], rtol=1e-8, atol=0)
    E = np.einsum("si,sij,sj->s", delta, Mu, delta) - 2 * np.einsum("si,si->s", delta, ru)
    assert np.allclose(E, -mlp.optimal_decrease(H, rhat) * s * s, rtol=1e-8, atol=0)


def test_block_jacobi_coordinates(small_problem):
    """H has identity diagonal blocks, and the output y = rhat is the block-Jacobi correction
    D^{-1} r_u on the unit (D = diag(M_aa, M_bb))."""
    P = small_problem
    Np = P.Np
    pairs, geom, _ = P.learned_units()
    Mu = mlp.unit_matrices(P.row_ptr, P.col, P.val, pairs)
    Xu, H = mlp.unit_transform(Mu)
    eye = np.eye(Np)
    assert np.abs(H[:, :Np, :Np] - eye).max() < 1e-10 and np.abs(H[:, Np:, Np:] - eye).max() < 1e-10
    rng = np.random.default_rng(4)
    r = rng.standard_normal(P.dof)
    X, rhat, s = mlp.unit_inputs(geom, pairs, r, Xu)
    delta = np.einsum("uji,uj->ui", Xu, rhat) * s[:, None]
    ru = np.concatenate([r.reshape(-1, Np)[pairs[:, 0]], r.reshape(-1, Np)[pairs[:, 1]]], axis=1)
    D = Mu.copy()
    D[:, :Np, Np:] = 0
    D[:, Np:, :Np] = 0
    assert np.allclose(delta, np.linalg.solve(D, ru[..., None])[..., 0], rtol=1e-8, atol=0)
    assert np.allclose(X[:, :geom.shape[1]], geom) and np.allclose(np.linalg.norm(rhat, axis=1), 1.0)
