"""Learned cut-cell correction: CUDA kernels against the FP64 oracle (oracle/mlp.py), training on
the GPU, and what the trained network gains.

Tolerances (FP32 arithmetic on the GPU against FP64 on the CPU, same FP32 inputs):
  * network forward, FP32 parameters: 1e-5 of the largest output; BF16 parameters (both
    sides rounded alike): 1e-5 as well
  * mean loss: 1e-4 relative; gradient: 1e-3 relative 2-norm (FP32 sums of up to a few
    hundred samples of 11k-parameter layers)
  * unit matrices in block-Jacobi coordinates (FP64 factorisation, FP32 copy): 1e-6 of the
    largest entry; samples (inputs, normalised residuals): 1e-5; optimal decreases c: 1e-4
    relative
  * one correction step: 1e-5 relative to the correction's norm; kept/rejected decisions equal
    wherever |E| exceeds 1e-3 of the largest |E| (elsewhere either decision is valid)
Gain: trained on problems with radii drawn from U(0.2, 0.4) (held-out radius excluded), the
network recovers more of the exact local solve's energy decrease on the held-out problem than
a block-Jacobi step on the same unit; the flexible-CG solve with the correction reaches the
oracle's solution within 1e-8 in about as many iterations as without it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from oracle import mlp as omlp  # noqa: E402
from paper_2003_02431_gb300 import learned, xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GAMMA, WLEV = 2, 2


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _bf16(a):
    """round-to-nearest-even to BF16, returned as float64"""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def _cfg(N, R, c=(0.5, 0.5, 0.5)):
    return xp.Config(D=3, N=N, k=2, c=c, R=R, muA=1, muB=1000, max_coarse_dof=300)


@pytest.fixture(scope="module")
def setup():
    P = xp.Problem(_cfg(14, 0.31, (0.48, 0.51, 0.5)))
    G = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=WLEV, low_precision=1)
    pairs, geom = learned.attach_units(G, P)
    O = oracle.Hierarchy(P, gamma=GAMMA)
    oracle.set_w_levels(O, WLEV)
    return P, G, O, pairs, geom


def test_forward_parity(setup):
    P, G, O, pairs, geom = setup
    net = learned.network_for(P, seed=7)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, net.n_in)).astype(np.float32)
    Xt = torch.from_numpy(X).to(DEV)
    theta = net.get_params().astype(np.float64)
    ref, _ = omlp.forward(theta, X.astype(np.float64), net.n_out)
    y = _n(net.forward(Xt, xdg.XDG_PREC_F32))
    assert np.abs(y - ref).max() < 1e-5 * np.abs(ref).max()
    refb, _ = omlp.forward(_bf16(theta), X.astype(np.float64), net.n_out)
    yb = _n(net.forward(Xt, xdg.XDG_PREC_BF16))
    assert np.abs(yb - refb).max() < 1e-5 * np.abs(refb).max()
    assert np.abs(refb - ref).max() > 0  # the BF16 path really rounds


def test_loss_and_gradient_parity(setup):
    P, G, O, pairs, geom = setup
    net = learned.network_for(P, seed=3)
    rng = np.random.default_rng(1)
    S, m = 257, 2 * P.Np
    X = rng.standard_normal((S, net.n_in)).astype(np.float32)
    A = rng.standard_normal((5, m, m))
    M = (np.einsum("uij,ukj->uik", A, A) + m * np.eye(m)).astype(np.float32)
    uid = rng.integers(0, 5, S).astype(np.int32)
    R = rng.standard_normal((S, m)).astype(np.float32)
    C = omlp.optimal_decrease(M[uid].astype(np.float64), R.astype(np.float64)).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)  # noqa: E731
    loss, g = net.loss_grad(t(X), t(uid), t(M), t(R), t(C))
    theta = net.get_params().astype(np.float64)
    ref_loss, ref_g = omlp.mean_loss_and_grad(theta, X.astype(np.float64), M[uid].astype(np.float64),
                                              R.astype(np.float64), C.astype(np.float64))
    assert abs(loss - ref_loss) < 1e-4 * abs(ref_loss)
    gg = _n(g).astype(np.float64)
    assert np.linalg.norm(gg - ref_g) < 1e-3 * np.linalg.norm(ref_g)


def test_unit_matrices_and_samples_parity(setup):
    P, G, O, pairs, geom = setup
    Np = P.Np
    Mu = omlp.unit_matrices(P.row_ptr, P.col, P.val, pairs)
    Xu, H = omlp.unit_transform(Mu)
    Ml = _n(G.units_local()).astype(np.float64)
    assert np.abs(Ml - H).max() <= 1e-6 * np.abs(H).max()
    b = P.b.reshape(-1)
    bt = torch.from_numpy(b.copy()).to(DEV)
    X, R, C = (_n(a) for a in G.units_samples(bt))
    import scipy.sparse as sp
    A = sp.bsr_matrix((P.val, P.col, P.row_ptr), shape=(P.dof, P.dof)).tocsr()
    z = O.vcycle(b)
    rp = b - A @ z
    Xr, rhat, s = omlp.unit_inputs(geom.astype(np.float64), pairs, rp, Xu)
    cref = omlp.optimal_decrease(H, rhat)
    assert np.abs(X - Xr).max() < 1e-5
    assert np.abs(R - rhat).max() < 1e-5
    assert np.all(np.abs(C - cref) <= 1e-4 * np.abs(cref) + 1e-30)


def test_learned_step_parity(setup):
    P, G, O, pairs, geom = setup
    Np = P.Np
    net = learned.network_for(P, seed=11)
    net.set_params(net.get_params() * 0.3)  # moderate corrections: both decisions occur
    G.learned_enable(net, theta=0.5)
    b = P.b.reshape(-1)
    z = O.vcycle(b)
    zt = torch.from_numpy(z.copy()).to(DEV)
    bt = torch.from_numpy(b.copy()).to(DEV)
    kept = G.learned_step(bt, zt)
    z1 = _n(zt)
    G.learned_enable(None)
    import scipy.sparse as sp
    A = sp.bsr_matrix((P.val, P.col, P.row_ptr), shape=(P.dof, P.dof)).tocsr()
    Mu = omlp.unit_matrices(P.row_ptr, P.col, P.val, pairs)
    theta = _bf16(net.get_params())
    zref, keep, E = omlp.learned_step(theta, geom.astype(np.float64), pairs, Mu, b - A @ z, z, 2 * Np, 0.5)
    assert 0 < keep.sum() < len(keep)
    unclear = np.abs(E) <= 1e-3 * np.abs(E).max()
    # blocks of units whose decision is not clear may differ; everything else must agree
    mask = np.ones(P.nb[0], bool)
    mask[pairs[unclear].reshape(-1)] = False
    d1, dr = z1.reshape(-1, Np)[mask], zref.reshape(-1, Np)[mask]
    dz = np.linalg.norm(dr - z.reshape(-1, Np)[mask])
    assert np.linalg.norm(d1 - dr) <= 1e-5 * max(dz, 1e-300)
    if not unclear.any():
        assert kept == int(keep.sum())


@pytest.fixture(scope="module")
def trained():
    """Network trained on 3 problems (radii from U(0.2, 0.4) away from the held-out 0.29)."""
    rng = np.random.Generator(np.random.PCG64(20030245))
    radii = []
    while len(radii) < 3:
        r = float(rng.uniform(0.2, 0.4))
        if abs(r - 0.29) > 0.005:
            radii.append(r)
    train = learned.SampleSet()
    keep = []
    for R in radii:
        P = xp.Problem(_cfg(14, R))
        G = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=WLEV, low_precision=1)
        learned.attach_units(G, P)
        b = torch.from_numpy(P.b.reshape(-1).copy()).to(DEV)
        train.add(G, learned.solver_residuals(G, b, 12))
        keep.append((P, G))
    net = learned.network_for(keep[0][0], seed=5)
    before = learned.evaluate(net, train)
    hist = learned.train(net, train, epochs=60, batch=256, lr=2e-3, seed=9)
    after = learned.evaluate(net, train)
    return net, before, hist, after


def test_training_lowers_the_loss(trained):
    net, before, hist, after = trained
    assert hist[-1] < hist[0]
    assert after < before
    assert after < -0.85, after  # >= 85 % of the exact local solve's decrease on the training data


def _block_jacobi_loss(ss):
    """mean loss of one block-Jacobi step on each unit (y = rhat) for the same samples"""
    X, uid, M, R, C = ss.tensors()
    M, R, C = M[uid.long()].double(), R.double(), C.double()
    L = (torch.einsum("si,sij,sj->s", R, M, R) - 2 * (R * R).sum(1)) / C
    return float(L.mean())


def test_gain_on_held_out_problem(trained):
    """What the trained network gains: on a held-out radius it recovers more of the exact local
    solve's energy decrease than a block-Jacobi step on the same unit does (measured: -0.93 vs
    -0.83 at 16^3). In the solve the correction keeps the accuracy and the iteration count
    within 2 (measured here: 53 against 52; the exact pair solve itself saves only about 2 of 52
    iterations: the slow modes of this multigrid are not local to the cut cells). Its wall time
    is not asserted: the three extra kernels per iteration cost about as much as the iterations
    saved (measured at 64^3: 61 instead of 65 iterations, 66.9 against 65.0 ms)."""
    net, *_ = trained
    P = xp.Problem(_cfg(16, 0.29))
    G = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=WLEV, low_precision=1)
    learned.attach_units(G, P)
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(DEV)
    held = learned.SampleSet()
    held.add(G, learned.solver_residuals(G, b, 8))
    loss, bj = learned.evaluate(net, held), _block_jacobi_loss(held)
    x0 = torch.zeros_like(b)
    plain = G.solve(b, x0, tol=1e-10, precision=xdg.XDG_PREC_F32)
    G.learned_enable(net, theta=0.25)
    x1 = torch.zeros_like(b)
    withnet = G.solve(b, x1, tol=1e-10, precision=xdg.XDG_PREC_F32)
    G.learned_enable(None)
    O = oracle.Hierarchy(P, gamma=GAMMA)
    oracle.set_w_levels(O, WLEV)
    xref, _, rr, _ = O.pcg(P.b, tol=1e-13, maxit=500)
    rel = np.linalg.norm(_n(x1) - xref) / np.linalg.norm(xref)
    print("held-out loss: network %.3f, block-Jacobi step %.3f; iterations plain %d, learned %d"
          % (loss, bj, plain["iterations"], withnet["iterations"]))
    assert loss < -0.8 and loss < bj - 0.05, (loss, bj)
    assert rel < 1e-8
    assert withnet["iterations"] <= plain["iterations"] + 2


def test_untrained_network_cannot_break_the_solve():
    """Fallback: corrections that would raise the error's energy are rejected unit by unit, so
    even a random network leaves the solve convergent and accurate."""
    P = xp.Problem(_cfg(14, 0.33, (0.49, 0.5, 0.52)))
    G = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=WLEV, low_precision=1)
    learned.attach_units(G, P)
    net = learned.network_for(P, seed=123)
    net.set_params(net.get_params() * 4.0)  # large random corrections
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(DEV)
    x0 = torch.zeros_like(b)
    plain = G.solve(b, x0, tol=1e-10, precision=xdg.XDG_PREC_F32)
    G.learned_enable(net, theta=0.25)
    z = torch.zeros_like(b)
    kept = G.learned_step(b, z)  # from z = 0 the residual is b
    x1 = torch.zeros_like(b)
    res = G.solve(b, x1, tol=1e-10, precision=xdg.XDG_PREC_F32)
    G.learned_enable(None)
    O = oracle.Hierarchy(P, gamma=GAMMA)
    oracle.set_w_levels(O, WLEV)
    xref, _, _, _ = O.pcg(P.b, tol=1e-13, maxit=500)
    assert np.linalg.norm(_n(x1) - xref) < 1e-8 * np.linalg.norm(xref)
    assert res["iterations"] <= int(1.2 * plain["iterations"]) + 2
    assert kept < G.n_units  # some corrections were rejected
