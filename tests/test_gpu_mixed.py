"""Mixed precision: FP32 / BF16 cycles inside FP64 flexible CG, against the FP64 oracle.

* apply with the stored FP32/BF16 operator vs the oracle's FP64 product with the same
  dequantised blocks (oracle.quantize_blocks) on the same FP32-rounded vector: elementwise
  within 1e-5 * (|A_q| |x|) -- FP32 accumulation over at most Np + nnz-per-row + 1 terms gives
  (Np + 40) * 6e-8 < 4e-6 of that bound
* one low-precision cycle stays close to the FP64 oracle's cycle (a preconditioner, not a
  parity claim): FP32 within 1e-3; BF16 (transfer blocks rounded to 8 bits, amplified by the
  ill-conditioned coarse levels: 2-5 % measured in 3D) within 1e-1
* the mixed solve reaches the FP64 oracle's solution within 1e-8 relative L2, as the FP64
  solve does, in a comparable number of iterations
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = {
    "2d_k2": (xp.config_2d_16(max_coarse_dof=60), 1),
    "2d_k4": (xp.Config(D=2, N=13, k=4, c=(0.5, 0.5, 0), R=0.27, muA=1, muB=10, max_coarse_dof=120), 2),
    "3d_k2": (xp.Config(D=3, N=14, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000, max_coarse_dof=300), 2),
    "3d_k3": (xp.Config(D=3, N=7, k=3, c=(0.48, 0.51, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=200), 1),
}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    cfg, gamma = CASES[request.param]
    P = xp.Problem(cfg)
    O = oracle.Hierarchy(P, gamma=gamma)
    G = xdg.Hierarchy.from_problem(P, gamma=gamma, low_precision=3)
    return request.param, P, O, G


@pytest.mark.parametrize("prec", [xdg.XDG_PREC_F32, xdg.XDG_PREC_BF16])
def test_apply_lowprec_matches_dequantised_oracle(case, prec):
    name, P, O, G = case
    rng = np.random.default_rng(31)
    for l in range(P.n_levels):
        lv = O.level(l)
        x = rng.standard_normal(lv["nb"] * P.Np)
        xf = x.astype(np.float32).astype(np.float64)
        q, _ = oracle.quantize_blocks(lv["val"], prec)
        ref = oracle.bsr_spmv(lv["row_ptr"], lv["col"], q, xf).reshape(-1)
        bound = oracle.bsr_spmv(lv["row_ptr"], lv["col"], np.abs(q), np.abs(xf)).reshape(-1)
        y = torch.empty(x.size, dtype=torch.float64, device=DEV)
        G.apply(l + 1, _t(x), y, prec=prec)
        assert np.all(np.abs(_n(y) - ref) <= 1e-5 * bound + 1e-300), (name, l, prec)


@pytest.mark.parametrize("prec,tol", [(xdg.XDG_PREC_F32, 1e-3), (xdg.XDG_PREC_BF16, 1e-1)])
def test_lowprec_cycle_close_to_fp64(case, prec, tol):
    name, P, O, G = case
    b = P.b.reshape(-1)
    ref = O.vcycle(b)
    x = torch.empty(P.dof, dtype=torch.float64, device=DEV)
    G.cycle(prec, _t(b), x)
    err = _rel(_n(x), ref)
    assert err < tol, (name, prec, err)


def test_split_row_mapping_agrees(case):
    """The two row mappings of the low-precision kernels (a row per group of Np lanes, or a row
    per warp split over its groups) compute the same operator apply up to FP32 summation order
    on every level, and cycles within the FP32 bound; the autotuned hierarchy reports which
    levels split."""
    name, P, O, G = case
    gamma = CASES[name][1]
    b = _t(P.b.reshape(-1))
    rng = np.random.default_rng(12)
    v = {l: _t(rng.standard_normal(P.nb[l - 1] * P.Np)) for l in range(1, P.n_levels + 1)}
    out = []
    for mode in (1, 2):
        H = xdg.Hierarchy.from_problem(P, gamma=gamma, low_precision=1, split_rows=mode)
        assert H.info()["split"] == [mode == 2] * P.n_levels
        x = torch.empty(P.dof, dtype=torch.float64, device=DEV)
        H.cycle(xdg.XDG_PREC_F32, b, x)
        ys = []
        for l in range(1, P.n_levels + 1):
            y = torch.empty_like(v[l])
            H.apply(l, v[l], y, prec=xdg.XDG_PREC_F32)
            ys.append(_n(y))
        out.append((_n(x), ys))
        H.destroy()
    # one apply: FP32 summation order only; a cycle amplifies rounding differences through the
    # ill-conditioned coarse levels as much as FP32 vs FP64 does (the 1e-3 bound above)
    for a, c in zip(out[0][1], out[1][1]):
        assert _rel(a, c) < 1e-6, name
    assert _rel(out[0][0], out[1][0]) < 1e-3, name
    assert _rel(out[1][0], O.vcycle(P.b.reshape(-1))) < 1e-3
    assert len(G.info()["split"]) == P.n_levels


@pytest.mark.parametrize("prec", [xdg.XDG_PREC_F32, xdg.XDG_PREC_BF16])
def test_fused_small_levels_match_launch_per_step(case, prec):
    """The small levels' V-cycle as one persistent launch (a cooperative grid, mode 2, or one
    thread-block cluster, mode 3) runs the same per-row arithmetic as the launch-per-step cycle:
    identical results, bit for bit (same row mapping on every side)."""
    name, P, O, G = case
    gamma = CASES[name][1]
    b = _t(P.b.reshape(-1))
    out = []
    for mode in (1, 2, 3):
        # the other creation-time choices pinned too, so that only the small levels' launch differs
        H = xdg.Hierarchy.from_problem(P, gamma=gamma, w_levels=1, low_precision=3, split_rows=1,
                                       fused_coarse=mode, outer_apply=2, symmetric=2)
        fused = H.info()["fused_level"]
        if mode >= 2 and P.n_levels >= 3 and P.nb[1] <= 16384:
            assert fused == 2, (name, fused)
            assert (H.info()["fused_cluster"] > 0) == (mode == 3)
        x = torch.empty(P.dof, dtype=torch.float64, device=DEV)
        H.cycle(prec, b, x)
        xs = torch.zeros_like(x)
        res = H.solve(b, xs, tol=1e-10, precision=prec)
        out.append((_n(x), _n(xs), res["iterations"], fused))
        H.destroy()
    assert out[0][3] == 0
    for k in (1, 2):
        assert np.array_equal(out[0][0], out[k][0]), (name, k)
        assert np.array_equal(out[0][1], out[k][1]) and out[0][2] == out[k][2], (name, k)


@pytest.mark.parametrize("prec", [xdg.XDG_PREC_F32, xdg.XDG_PREC_BF16])
def test_mixed_solve_reaches_fp64_oracle_solution(case, prec):
    name, P, O, G = case
    ref, it_o, _, _ = O.pcg(P.b, tol=1e-14, maxit=600)
    _, it64, _, _ = O.pcg(P.b, tol=1e-11, maxit=600)
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve(_t(P.b), x, tol=1e-11, maxit=600, precision=prec)
    assert info["relres"] <= 1e-11
    assert _rel(_n(x), ref) < 1e-8, (name, prec, info)
    assert info["iterations"] <= 1.5 * it64 + 3, (info["iterations"], it64)


def test_mixed_requires_stored_copy():
    P = xp.Problem(xp.config_2d_16(max_coarse_dof=60))
    G = xdg.Hierarchy.from_problem(P)  # no low-precision copies
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    with pytest.raises(xdg.XdgError) as e:
        G.solve(_t(P.b), x, precision=xdg.XDG_PREC_BF16)
    assert e.value.code == xdg.XDG_EINVAL


def test_full_size_mixed_solves():
    """3D 64^3 workload: both mixed solves reach the FP64 oracle's solution within 1e-8."""
    P = xp.Problem(xp.config_3d_64(max_coarse_dof=1000))
    O = oracle.Hierarchy(P, gamma=2)
    ref, _, _, _ = O.pcg(P.b, tol=1e-14, maxit=400)
    G = xdg.Hierarchy.from_problem(P, gamma=2, low_precision=3)
    for prec in (xdg.XDG_PREC_F32, xdg.XDG_PREC_BF16):
        x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
        info = G.solve(_t(P.b), x, tol=1e-10, maxit=400, precision=prec)
        assert _rel(_n(x), ref) < 1e-8, (prec, info)
