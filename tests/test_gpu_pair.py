"""The level-1 apply from FP32 pairs (XDG_PREC_F64_PAIR) against the oracle's FP64 product.

Error bound per output entry i, from the arithmetic (u = 2^-24, the FP32 unit roundoff):
  * splitting each operator and vector entry into scaled hi + lo FP32 numbers leaves at most
    u^2 relative error per entry; dropping lo*lo another u^2: 3 u^2 per product
  * the three cross products accumulated by fused multiply-adds into the product's rounding
    error e: at most 6 u^2 per product
  * TwoSum keeps the running sum's errors exactly; their FP32 sum over the 2 Np values of one
    block adds at most sum_k u (4 k u) T <= 2 Np^2 u^2 T (T: the block's sum |a||x|)
  * the blocks' results (hi + lo) are scaled by powers of two (exact) and summed in FP64: at
    most 2 nnz_row 2^-53 of the row's sum |a||x|
so |y_pair - y|_i <= ((9 + 2 Np^2) u^2 + 64 * 2^-53) (|M||x|)_i, with the oracle's own FP64
rounding (at most (Np nnz_row) 2^-53, inside the last term's slack for these sizes) beside it.
The test asserts that bound, the 1e-12 norm-wise bound of the FP64 apply test, the range
handling (vector blocks scaled by 2^+-600, zero blocks), and that a mixed-precision solve with
the pair product reaches the oracle's solution as the FP64 outer apply does.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U2 = 2.0 ** -48

CASES = {
    "2d_k2": xp.config_2d_16(max_coarse_dof=60),                                       # Np = 6
    "2d_k4": xp.Config(D=2, N=13, k=4, c=(0.5, 0.5, 0), R=0.27, muA=1, muB=10, max_coarse_dof=120),  # 15
    "3d_k2": xp.Config(D=3, N=14, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000, max_coarse_dof=300),  # 10
    "3d_k3": xp.Config(D=3, N=7, k=3, c=(0.48, 0.51, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=200),  # 20
}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    P = xp.Problem(CASES[request.param])
    G = xdg.Hierarchy.from_problem(P, gamma=2, low_precision=1, outer_apply=2)
    return request.param, P, G


def _check(P, G, x):
    ref = oracle.bsr_spmv(P.row_ptr, P.col, P.val, x).reshape(-1)
    mag = oracle.bsr_spmv(P.row_ptr, P.col, np.abs(P.val), np.abs(x)).reshape(-1)
    y = torch.empty(P.dof, dtype=torch.float64, device=DEV)
    G.apply(1, _t(x), y, prec=xdg.XDG_PREC_F64_PAIR)
    got = _n(y)
    bound = ((9 + 2 * P.Np ** 2) * U2 + 64 * 2.0 ** -53) * mag
    err = np.abs(got - ref)
    assert np.all(err <= bound), (float((err / np.maximum(bound, 1e-300)).max()))
    return got, ref


def test_pair_apply_within_bound(case):
    name, P, G = case
    assert G.info()["outer_pair"]
    rng = np.random.default_rng(5)
    x = rng.standard_normal(P.dof)
    got, ref = _check(P, G, x)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12, name


def test_pair_apply_range_and_zero_blocks(case):
    name, P, G = case
    rng = np.random.default_rng(6)
    nb = P.nb[0]
    x = rng.standard_normal((nb, P.Np))
    # block magnitudes spread over 2^-600 .. 2^600 (the per-block exponents absorb them) and
    # whole zero blocks
    x *= np.exp2(rng.integers(-600, 601, nb)).reshape(-1, 1)
    x[rng.random(nb) < 0.1] = 0.0
    _check(P, G, x.reshape(-1))
    # a vector scaled as a whole: the product scales exactly
    x2 = rng.standard_normal(P.dof)
    y1 = torch.empty(P.dof, dtype=torch.float64, device=DEV)
    y2 = torch.empty_like(y1)
    G.apply(1, _t(x2), y1, prec=xdg.XDG_PREC_F64_PAIR)
    G.apply(1, _t(x2 * 2.0 ** -700), y2, prec=xdg.XDG_PREC_F64_PAIR)
    assert np.array_equal(_n(y1) * 2.0 ** -700, _n(y2))
    z = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    G.apply(1, z, y1, prec=xdg.XDG_PREC_F64_PAIR)
    assert not np.any(_n(y1))


def test_pair_needs_its_copy_and_level_1(case):
    name, P, G = case
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    y = torch.empty_like(x)
    with pytest.raises(xdg.XdgError):
        G.apply(2, x[:P.nb[1] * P.Np], y[:P.nb[1] * P.Np], prec=xdg.XDG_PREC_F64_PAIR)
    H = xdg.Hierarchy.from_problem(P, gamma=2, low_precision=1, outer_apply=1)
    assert not H.info()["outer_pair"]
    with pytest.raises(xdg.XdgError):
        H.apply(1, x, y, prec=xdg.XDG_PREC_F64_PAIR)
    H.destroy()


def test_mixed_solve_with_pair_apply_reaches_oracle_solution(case):
    name, P, G = case
    O = oracle.Hierarchy(P, gamma=2)
    xref, _, rr, _ = O.pcg(P.b, tol=1e-13, maxit=500)
    O.close()
    assert rr < 1e-12
    H = xdg.Hierarchy.from_problem(P, gamma=2, low_precision=1, outer_apply=1)
    b = _t(P.b)
    its = []
    for hier in (G, H):
        x = torch.zeros_like(b)
        info = hier.solve(b, x, tol=1e-10, maxit=300, precision=xdg.XDG_PREC_F32)
        assert info["relres"] < 1e-10
        xs = _n(x)
        assert np.linalg.norm(xs - xref.reshape(-1)) / np.linalg.norm(xref) < 1e-8, name
        its.append(info["iterations"])
    assert abs(its[0] - its[1]) <= 1, its
    H.destroy()


def test_batched_solve_with_pair_apply():
    """A batch whose flexible CG applies M from FP32 pairs (rows of finished problems skipped)
    reaches every problem's oracle solution, in the iterations of the FP64 outer apply (+-1)."""
    probs = [xp.Problem(c) for c in xp.batch_configs(5, seed=21, N_range=(9, 18), ks=(2, 3, 4), max_levels=4)]
    bb = _t(np.concatenate([p.b.reshape(-1) for p in probs]))
    its = {}
    for mode in (2, 1):
        bt = xdg.Batch(probs, gamma=2, low_precision=1, outer_apply=mode)
        x = torch.zeros_like(bb)
        res = bt.solve(bb, x, tol=1e-10, maxit=300, precision=xdg.XDG_PREC_F32)
        xs, off = _n(x), bt.offsets
        for i, p in enumerate(probs):
            assert res["problems"][i]["status"] == xdg.XDG_OK
            if mode == 2:
                O = oracle.Hierarchy(p, gamma=2)
                xref, _, rr, _ = O.pcg(p.b, tol=1e-13, maxit=500)
                O.close()
                assert rr < 1e-12
                err = np.linalg.norm(xs[off[i]:off[i + 1]] - xref.reshape(-1)) / np.linalg.norm(xref)
                assert err < 1e-8, (i, err)
        its[mode] = [r["iterations"] for r in res["problems"]]
        bt.destroy()
    assert all(abs(a - b) <= 1 for a, b in zip(its[2], its[1])), its
