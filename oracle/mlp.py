"""Oracle of the learned cut-cell correction (plain FP64 numpy).

TEST INFRASTRUCTURE ONLY: imported by the tests (and nothing in the CUDA library).

The learned smoother is not part of arXiv 2003.02431; it extends the paper's smoothing step
(the cell-local dense solves of Algorithm 1 and the block Schwarz smoother, sec. 3.3) with a
correction on the two species blocks of every cut background cell (a "unit": the pair of
level-1 blocks that hold the A and B parts of one cut cell). What the correction should be
follows from the energy norm the multigrid method is built on: for a correction delta
supported on the unit u, the true error e of the current iterate (r = M e) changes its
energy by

    ||e - delta||_M^2 - ||e||_M^2 = delta^T M_uu delta - 2 delta^T r_u,

minimised by the exact local solve delta* = M_uu^{-1} r_u with value -r_u^T M_uu^{-1} r_u.
The unit works in the coordinates of the block-Jacobi smoother: with X_a = L_a^{-1},
X_b = L_b^{-1} the inverse Cholesky factors of the diagonal blocks M_aa = L_a L_a^T,
M_bb = L_b L_b^T and Xu = diag(X_a, X_b),

    rt = Xu r_u,   H = Xu M_uu Xu^T (identity diagonal blocks),   delta = s Xu^T y,

with s = ||rt||_2, rhat = rt / s and y the network output; then the energy change is
s^2 (y^T H y - 2 y^T rhat), the exact local solve is y* = H^{-1} rhat (of order one), and
y = rhat is one block-Jacobi step on the unit. The training loss of one sample is the energy
change divided by its optimal value s^2 c, c = rhat^T H^{-1} rhat, so that -1 means the network
reproduces the local solve and 0 means no gain:

    L = (y^T H y - 2 y^T rhat) / c.

Network: n_in inputs -> 3 hidden layers of width 64 with GELU (exact, erf form) -> n_out =
2 Np outputs. Flat parameter layout (row-major): W1[n_in][64], b1[64], W2[64][64], b2[64],
W3[64][64], b3[64], W4[64][n_out], b4[n_out]; a layer computes a_out = act(a_in W + b).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

WIDTH = 64


def layout(n_in: int, n_out: int, width: int = WIDTH):
    """[(name, shape, offset)] of the flat parameter vector."""
    shapes = [("W1", (n_in, width)), ("b1", (width,)), ("W2", (width, width)), ("b2", (width,)),
              ("W3", (width, width)), ("b3", (width,)), ("W4", (width, n_out)), ("b4", (n_out,))]
    out, off = [], 0
    for name, shp in shapes:
        out.append((name, shp, off))
        off += int(np.prod(shp))
    return out, off


def unpack(theta, n_in, n_out):
    lay, total = layout(n_in, n_out)
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == total
    return {name: theta[off:off + int(np.prod(shp))].reshape(shp) for name, shp, off in lay}


def gelu(x):
    """x Phi(x), Phi the standard normal distribution function."""
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    """d/dx x Phi(x) = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(theta, X, n_out):
    """Y = network(X) for samples X [S][n_in]; returns (Y, cache of pre-activations)."""
    X = np.asarray(X, dtype=np.float64)
    p = unpack(theta, X.shape[1], n_out)
    a0 = X
    z1 = a0 @ p["W1"] + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"] + p["b2"]
    a2 = gelu(z2)
    z3 = a2 @ p["W3"] + p["b3"]
    a3 = gelu(z3)
    Y = a3 @ p["W4"] + p["b4"]
    return Y, (a0, z1, a1, z2, a2, z3, a3)


def loss(Y, M, R, c):
    """Per-sample loss (y^T M y - 2 y^T r) / c and its gradient with respect to y."""
    MY = np.einsum("sij,sj->si", M, Y)
    L = (np.einsum("si,si->s", Y, MY) - 2.0 * np.einsum("si,si->s", Y, R)) / c
    dY = 2.0 * (MY - R) / c[:, None]
    return L, dY


def backward(theta, cache, dY, n_out):
    """Gradient of sum_s w_s L_s for the upstream gradient dY [S][n_out] (flat vector)."""
    a0, z1, a1, z2, a2, z3, a3 = cache
    p = unpack(theta, a0.shape[1], n_out)
    g = {}
    g["W4"] = a3.T @ dY
    g["b4"] = dY.sum(0)
    d3 = (dY @ p["W4"].T) * gelu_grad(z3)
    g["W3"] = a2.T @ d3
    g["b3"] = d3.sum(0)
    d2 = (d3 @ p["W3"].T) * gelu_grad(z2)
    g["W2"] = a1.T @ d2
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"].T) * gelu_grad(z1)
    g["W1"] = a0.T @ d1
    g["b1"] = d1.sum(0)
    lay, total = layout(a0.shape[1], n_out)
    out = np.zeros(total)
    for name, shp, off in lay:
        out[off:off + int(np.prod(shp))] = g[name].reshape(-1)
    return out


def mean_loss_and_grad(theta, X, M, R, c):
    """Mean loss over the samples and its gradient with respect to the parameters."""
    n_out = R.shape[1]
    Y, cache = forward(theta, X, n_out)
    L, dY = loss(Y, M, R, c)
    S = X.shape[0]
    return L.mean(), backward(theta, cache, dY / S, n_out)


# ------------------------------------------------------------------------------------------
# units of a problem
def unit_pairs(cut_cells):
    """Distinct (A block, B block) pairs of the cut cells, in order of their first cell;
    also the first cell of every pair (its geometry describes the unit)."""
    seen, pairs, cells = set(), [], []
    for cell, a, b in np.asarray(cut_cells):
        key = (int(a), int(b))
        if key not in seen:
            seen.add(key)
            pairs.append(key)
            cells.append(int(cell))
    return np.array(pairs, dtype=np.int32).reshape(-1, 2), np.array(cells, dtype=np.int32)


def unit_matrices(row_ptr, col, val, pairs):
    """M_uu = [[M_aa, M_ab], [M_ba, M_bb]] of every unit from the level-1 BSR operator."""
    Np = val.shape[-1]

    def block(i, j):
        for z in range(row_ptr[i], row_ptr[i + 1]):
            if col[z] == j:
                return val[z]
        return np.zeros((Np, Np))

    out = np.zeros((len(pairs), 2 * Np, 2 * Np))
    for u, (a, b) in enumerate(pairs):
        out[u, :Np, :Np] = block(a, a)
        out[u, :Np, Np:] = block(a, b)
        out[u, Np:, :Np] = block(b, a)
        out[u, Np:, Np:] = block(b, b)
    return out


def unit_transform(Mu):
    """Xu = diag(L_a^{-1}, L_b^{-1}) and H = Xu M_uu Xu^T of every unit."""
    U, m, _ = Mu.shape
    Np = m // 2
    Xu = np.zeros_like(Mu)
    for u in range(U):
        for h in range(2):
            sl = slice(h * Np, (h + 1) * Np)
            Lh = np.linalg.cholesky(Mu[u, sl, sl])
            Xu[u, sl, sl] = np.linalg.inv(Lh)
    H = np.einsum("uij,ujk,ulk->uil", Xu, Mu, Xu)
    return Xu, 0.5 * (H + H.transpose(0, 2, 1))


def unit_inputs(geom, pairs, r, Xu):
    """Network inputs [geom, rhat], rhat and s of every unit for the residual r
    (rt = Xu [r_a; r_b], s = ||rt||, rhat = rt / s)."""
    Np = Xu.shape[1] // 2
    ru = np.concatenate([r.reshape(-1, Np)[pairs[:, 0]], r.reshape(-1, Np)[pairs[:, 1]]], axis=1)
    rt = np.einsum("uij,uj->ui", Xu, ru)
    s = np.linalg.norm(rt, axis=1)
    s_safe = np.where(s > 0, s, 1.0)
    rhat = rt / s_safe[:, None]
    return np.concatenate([geom, rhat], axis=1), rhat, s


def optimal_decrease(H, rhat):
    """c = rhat^T H^{-1} rhat per unit."""
    return np.einsum("si,si->s", rhat, np.linalg.solve(H, rhat[..., None])[..., 0])


def learned_step(theta, geom, pairs, Mu, r_after, z, n_out, theta_damp):
    """z + theta_damp * sum over accepted units of delta_u, for the residual r_after = r - M z
    of the cycle's result z. A unit's correction delta = s Xu^T network(inputs) is accepted when
    it lowers the energy of the error: E = delta^T M_uu delta - 2 delta^T r_u < 0."""
    Np = n_out // 2
    Xu, H = unit_transform(Mu)
    X, rhat, s = unit_inputs(geom, pairs, r_after, Xu)
    Y, _ = forward(theta, X, n_out)
    delta = np.einsum("uji,uj->ui", Xu, Y) * s[:, None]
    ru = np.concatenate([r_after.reshape(-1, Np)[pairs[:, 0]], r_after.reshape(-1, Np)[pairs[:, 1]]], axis=1)
    E = np.einsum("si,sij,sj->s", delta, Mu, delta) - 2.0 * np.einsum("si,si->s", delta, ru)
    keep = (E < 0) & (s > 0)
    out = z.reshape(-1, Np).copy()
    for u in np.nonzero(keep)[0]:
        a, b = pairs[u]
        out[a] += theta_damp * delta[u, :Np]
        out[b] += theta_damp * delta[u, Np:]
    return out.reshape(-1), keep, E
