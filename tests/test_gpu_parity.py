"""Parity of the CUDA path (libxdg through its C ABI) with the CPU oracle.

Tolerances (FP64 on both sides; the two differ only by summation order, fused multiply-adds
and explicit inverses against Cholesky substitutions), checked entry by entry (tests/_bounds.py
derives each bound):
  * operator apply: |y_i - ref_i| <= 2 (n_i + 2) u (|M||x|)_i, n_i the terms of row i
  * restriction, prolongation: the same with |R|^T (|b| + |M||x|) and |x| + |R||z_c|
  * smoothing step: the residual as above plus the componentwise error of the block solves,
    c Np u |D^-1||L||L^T||D^-1||r| per block
  * Galerkin coarse operators: identical sparsity, values within 1e-12 of the largest entry
  * coarsest-level solve: 1e-12 relative to the solution times max(1, cond/1e4) (an explicit
    inverse and a triangular solve differ by about cond * eps)
  * one multigrid cycle: every block within 1e-9 of its own largest entry (a block that
    cancels to a small fraction of its neighbours carries their rounding), and 1e-12
    relative in the 2-norm
  * the 2-norm checks of the smoothing step and the cycle (1e-12) scale with Np / 20 above
    Np = 20: they contain explicit block inverses compared with Cholesky substitutions, whose
    difference grows with the block size (gamma_Np); the entry-wise bounds are not scaled. The
    cycle's check also carries the coarsest solve's allowance, max(1, cond/1e4) (an explicit
    inverse against a triangular solve, as in the coarsest-solve check)
  * solution of the multigrid-preconditioned CG: 1e-8 relative L2 (coefficient 2-norm, the
    bases are orthonormal) against the oracle's solution converged to 1e-14
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from _bounds import (SmoothBound, apply_bound, check, check_blocks, prolong_bound,  # noqa: E402
                     restrict_bound)
from conftest import dense_from_bsr  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

CASES = {
    # name: (config, gamma)
    "2d_k2_c1": (xp.config_2d_16(max_coarse_dof=60), 1),
    "2d_k3": (xp.Config(D=2, N=24, k=3, c=(0.46, 0.53, 0), R=0.31, muA=1, muB=100, max_coarse_dof=120), 2),
    "2d_k4": (xp.Config(D=2, N=13, k=4, c=(0.5, 0.5, 0), R=0.27, muA=1, muB=10, max_coarse_dof=120), 1),
    "3d_k2": (xp.Config(D=3, N=14, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000, max_coarse_dof=300), 2),
    "3d_k3": (xp.Config(D=3, N=7, k=3, c=(0.48, 0.51, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=200), 1),
    # W-cycle on the finest level only, V-cycle below
    "3d_k2_w1": (xp.Config(D=3, N=12, k=2, c=(0.47, 0.52, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=100), 2, 1),
    # blocks wider than a warp (Np = 35, 56): the warp-per-row kernels
    "3d_k4": (xp.Config(D=3, N=7, k=4, c=(0.48, 0.51, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=600), 2),
    "3d_k5": (xp.Config(D=3, N=6, k=5, c=(0.48, 0.51, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=600), 1),
}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _norm_tol(Np):
    """2-norm tolerance of the steps with block inverses (smoothing, cycle)."""
    return 1e-12 * max(1.0, Np / 20.0)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    cfg, gamma, *rest = CASES[request.param]
    wlev = rest[0] if rest else 0
    P = xp.Problem(cfg)
    assert P.n_levels >= 2
    O = oracle.Hierarchy(P, gamma=gamma)
    if wlev:
        oracle.set_w_levels(O, wlev)
    G = xdg.Hierarchy.from_problem(P, gamma=gamma, w_levels=wlev)
    return request.param, P, O, G


def test_apply_parity(case):
    name, P, O, G = case
    rng = np.random.default_rng(1)
    for l in range(P.n_levels):
        lv = O.level(l)
        n = lv["nb"] * P.Np
        x = rng.standard_normal(n)
        ref = oracle.bsr_spmv(lv["row_ptr"], lv["col"], lv["val"], x).reshape(-1)
        y = torch.empty(n, dtype=torch.float64, device=DEV)
        G.apply(l + 1, _t(x), y)
        got = _n(y)
        check(got, ref, apply_bound(lv["row_ptr"], lv["col"], lv["val"], x), (name, l))
        assert _rel(got, ref) < 1e-12, (name, l)


def test_galerkin_operators_parity(case):
    name, P, O, G = case
    for l in range(P.n_levels):
        lv = O.level(l)
        rp, cl, vl = G.export_level(l + 1)
        assert np.array_equal(rp, lv["row_ptr"]) and np.array_equal(cl, lv["col"]), (name, l)
        assert np.abs(vl - lv["val"]).max() <= 1e-12 * np.abs(lv["val"]).max(), (name, l)


def test_damping_estimates_parity(case):
    name, P, O, G = case
    inf = G.info()
    for l in range(P.n_levels - 1):
        lv = O.level(l)
        assert abs(inf["lambda_max"][l] - lv["lmax"]) <= 1e-10 * lv["lmax"], (name, l)
        assert abs(inf["omega"][l] - lv["omega"]) <= 1e-10 * lv["omega"]


def test_smoother_parity(case):
    name, P, O, G = case
    rng = np.random.default_rng(2)
    for l in range(P.n_levels - 1):
        lv = O.level(l)
        G.set_damping(l + 1, lv["omega"])  # the same damping on both sides
        bound = SmoothBound(lv)
        n = lv["nb"] * P.Np
        b, x = rng.standard_normal(n), rng.standard_normal(n)
        ref = O.smooth(l, b, x)
        out = torch.empty(n, dtype=torch.float64, device=DEV)
        G.smooth(l + 1, _t(b), _t(x), out)
        check(_n(out), ref, bound(lv["omega"], b, x), (name, l))
        assert _rel(_n(out), ref) < _norm_tol(P.Np), (name, l)
        # from a zero initial guess
        ref0 = O.smooth(l, b, np.zeros(n))
        G.smooth(l + 1, _t(b), None, out)
        check(_n(out), ref0, bound(lv["omega"], b, np.zeros(n)), (name, l, "x=0"))
        assert _rel(_n(out), ref0) < _norm_tol(P.Np)


def test_transfer_parity(case):
    name, P, O, G = case
    rng = np.random.default_rng(3)
    for l in range(P.n_levels - 1):
        lv = O.level(l)
        n, nc = lv["nb"] * P.Np, P.nb[l + 1] * P.Np
        b, x, zc = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(nc)
        r = b - oracle.bsr_spmv(lv["row_ptr"], lv["col"], lv["val"], x).reshape(-1)
        ref = oracle.restrict(P.agg[l], P.R[l], r, P.nb[l + 1]).reshape(-1)
        rc = torch.empty(nc, dtype=torch.float64, device=DEV)
        G.restrict(l + 1, _t(b), _t(x), rc)
        check(_n(rc), ref, restrict_bound(lv["row_ptr"], lv["col"], lv["val"], P.agg[l], P.R[l], b, x, P.nb[l + 1]),
              (name, l))
        assert _rel(_n(rc), ref) < 1e-12, (name, l)
        G.restrict(l + 1, _t(b), None, rc)
        ref_b = oracle.restrict(P.agg[l], P.R[l], b, P.nb[l + 1]).reshape(-1)
        check(_n(rc), ref_b, restrict_bound(None, None, None, P.agg[l], P.R[l], b, None, P.nb[l + 1]), (name, l))
        refp = oracle.prolong_add(P.agg[l], P.R[l], zc, x).reshape(-1)
        pb = prolong_bound(P.agg[l], P.R[l], zc, x)
        xo = torch.empty(n, dtype=torch.float64, device=DEV)
        G.prolong(l + 1, _t(zc), _t(x), xo)
        check(_n(xo), refp, pb, (name, l))
        xi = _t(x)
        G.prolong(l + 1, _t(zc), xi, xi)  # in place
        check(_n(xi), refp, pb, (name, l, "in place"))


def test_coarse_solve_parity(case):
    name, P, O, G = case
    lv = O.level(P.n_levels - 1)
    A = dense_from_bsr(lv["row_ptr"], lv["col"], lv["val"])
    cond = np.linalg.cond(A)
    r = np.random.default_rng(4).standard_normal(A.shape[0])
    ref = O.coarse_solve(r)
    z = torch.empty_like(_t(r))
    G.coarse_solve(_t(r), z)
    assert _rel(_n(z), ref) < 1e-12 * max(1.0, cond / 1e4), (name, cond)


def test_cycle_parity(case):
    """One cycle with the same damping on both sides (the Lanczos estimates themselves agree to
    the 1e-10 of test_damping_estimates_parity, and a cycle is about as sensitive to the damping
    as its relative size)."""
    name, P, O, G = case
    for l in range(P.n_levels - 1):
        G.set_damping(l + 1, O.level(l)["omega"])
    lc = O.level(P.n_levels - 1)
    cond = np.linalg.cond(dense_from_bsr(lc["row_ptr"], lc["col"], lc["val"]))
    tol = _norm_tol(P.Np) * max(1.0, cond / 1e4)
    rng = np.random.default_rng(5)
    for b in (P.b.reshape(-1), rng.standard_normal(P.dof)):
        ref = O.vcycle(b)
        x = torch.empty(P.dof, dtype=torch.float64, device=DEV)
        bt = _t(b)
        G.vcycle(bt, x)
        got = _n(x)
        check_blocks(got, ref, P.Np, 1e-9, name)
        assert _rel(got, ref) < tol, (name, cond)
        G.vcycle(bt, x)  # graph replay gives the same result
        assert np.array_equal(_n(x), got)


def test_solve_parity(case):
    name, P, O, G = case
    ref, it, rr, _ = O.pcg(P.b, tol=1e-14, maxit=600)
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve(_t(P.b), x, tol=1e-11, maxit=600)
    assert info["relres"] <= 1e-11
    assert _rel(_n(x), ref) < 1e-8, (name, info)
    # iteration counts of the two implementations agree closely
    _, it_o, _, _ = O.pcg(P.b, tol=1e-11, maxit=600)
    assert abs(info["iterations"] - it_o) <= 2, (info["iterations"], it_o)


def test_solve_host_path(case):
    name, P, O, G = case
    ref, _, _, _ = O.pcg(P.b, tol=1e-14, maxit=600)
    b = torch.from_numpy(P.b.reshape(-1).copy()).pin_memory().numpy()
    x = torch.zeros(P.dof, dtype=torch.float64).pin_memory().numpy()
    info = G.solve_host(b, x, tol=1e-11, maxit=600)
    assert _rel(x, ref) < 1e-8 and info["relres"] <= 1e-11


# ----------------------------------------------------------------------------- edge cases
def test_single_level_direct_solve():
    P = xp.Problem(xp.Config(D=2, N=5, k=2, c=(0.5, 0.5, 0), R=0.3, max_levels=1))
    G = xdg.Hierarchy.from_problem(P)
    A = dense_from_bsr(P.row_ptr, P.col, P.val)
    ref = np.linalg.solve(A, P.b.reshape(-1))
    x = torch.empty(P.dof, dtype=torch.float64, device=DEV)
    G.vcycle(_t(P.b), x)
    assert _rel(_n(x), ref) < 1e-10
    xs = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve(_t(P.b), xs, tol=1e-12)
    assert info["iterations"] <= 2 and _rel(_n(xs), ref) < 1e-10


@pytest.fixture(scope="module")
def small():
    P = xp.Problem(xp.config_2d_16(max_coarse_dof=60))
    return P, xdg.Hierarchy.from_problem(P)


def test_zero_rhs_and_exact_initial_guess(small):
    P, G = small
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve(torch.zeros(P.dof, dtype=torch.float64, device=DEV), x, tol=1e-10)
    assert info["iterations"] == 0 and float(x.abs().max()) == 0.0
    ref, _, _, _ = oracle.Hierarchy(P).pcg(P.b, tol=1e-14)
    x = _t(ref)
    info = G.solve(_t(P.b), x, tol=1e-10)
    assert info["iterations"] == 0


def test_iteration_limit_and_resume(small):
    P, G = small
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve(_t(P.b), x, tol=1e-12, maxit=3, raise_on_error=False)
    assert info["status"] == xdg.XDG_ENOTCONV and info["iterations"] == 3
    info2 = G.solve(_t(P.b), x, tol=1e-12, maxit=500)  # resume from the partial iterate
    assert info2["status"] == xdg.XDG_OK and info2["relres"] <= 1e-12


def test_time_budget(small):
    P, G = small
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve(_t(P.b), x, tol=1e-14, maxit=500, time_budget_ms=1e-9, raise_on_error=False)
    assert info["status"] == xdg.XDG_ETIMEOUT and info["iterations"] >= 1
    # the context stays usable
    info = G.solve(_t(P.b), x, tol=1e-10, maxit=500)
    assert info["status"] == xdg.XDG_OK


def test_rejects_invalid_inputs():
    P = xp.Problem(xp.config_2d_16(max_coarse_dof=60))
    base = dict(Np=P.Np, nb=P.nb, row_ptr=P.row_ptr, col=P.col, val=P.val, aggs=P.agg, Rs=P.R)

    def make(**over):
        kw = dict(base)
        kw.update(over)
        return xdg.Hierarchy(**kw)

    col = P.col.copy()
    col[5] = P.nb[0] + 3
    with pytest.raises(xdg.XdgError) as e:
        make(col=col)
    assert e.value.code == xdg.XDG_EINVAL
    agg = [a.copy() for a in P.agg]
    agg[0][0] = -1
    with pytest.raises(xdg.XdgError) as e:
        make(aggs=agg)
    assert e.value.code == xdg.XDG_EINVAL
    val = P.val.copy()
    val[0, 0, 0] = np.nan
    with pytest.raises(xdg.XdgError) as e:
        make(val=val)
    assert e.value.code == xdg.XDG_EINVAL
    with pytest.raises(xdg.XdgError) as e:
        make(Np=7)
    assert e.value.code == xdg.XDG_EINVAL
    # a negative definite operator: its diagonal blocks have no Cholesky factor
    with pytest.raises(xdg.XdgError) as e:
        make(val=-P.val)
    assert e.value.code == xdg.XDG_EBREAKDOWN


# ----------------------------------------------------------------------------- full size
_C2_REF = {}


@pytest.fixture(scope="module")
def c2():
    """3D, 64^3 cells, sphere R=0.31, mu 1:1000, k=2: about 2.66 million DOF."""
    P = xp.Problem(xp.config_3d_64(max_coarse_dof=1000))
    O = oracle.Hierarchy(P, gamma=2)
    G = xdg.Hierarchy.from_problem(P, gamma=2)
    return P, O, G


def _c2_solution(P, O):
    """The oracle's solution of the 64^3 system (PCG to 1e-14), computed once."""
    if "x" not in _C2_REF:
        ref, it, rr, _ = O.pcg(P.b, tol=1e-14, maxit=400)
        assert rr < 1e-13
        _C2_REF["x"] = ref
    return _C2_REF["x"]


def test_full_size_apply_cycle_parity(c2):
    P, O, G = c2
    x = np.random.default_rng(6).standard_normal(P.dof)
    y = torch.empty(P.dof, dtype=torch.float64, device=DEV)
    G.apply(1, _t(x), y)
    ref = oracle.bsr_spmv(P.row_ptr, P.col, P.val, x).reshape(-1)
    check(_n(y), ref, apply_bound(P.row_ptr, P.col, P.val, x), "apply 64^3")
    assert _rel(_n(y), ref) < 1e-12
    for l in range(P.n_levels - 1):  # same damping on both sides (see test_cycle_parity)
        G.set_damping(l + 1, O.level(l)["omega"])
    z = torch.empty(P.dof, dtype=torch.float64, device=DEV)
    G.vcycle(_t(P.b), z)
    refz = O.vcycle(P.b)
    check_blocks(_n(z), refz, P.Np, 1e-9, "cycle 64^3")
    assert _rel(_n(z), refz) < 1e-12


def test_full_size_solve_parity(c2):
    P, O, G = c2
    ref = _c2_solution(P, O)
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve(_t(P.b), x, tol=1e-11, maxit=400)
    assert _rel(_n(x), ref) < 1e-8, info


def test_full_size_benchmark_configuration(c2):
    """The benchmark's exact configuration at 64^3: W-cycle on the two finest levels, V below;
    creation-time autotuning of the outer apply (FP32 pairs), the level-1 symmetric storage,
    the split-row mapping and the fused small levels; FP32 cycle inside FP64 flexible CG, and
    the plain FP64 and BF16-transfer paths, each to the benchmark's 1e-10 relative residual.
    Every solution lies within 1e-8 relative L2 of the oracle's."""
    P, O, _ = c2
    ref = _c2_solution(P, O)
    H = xdg.Hierarchy.from_problem(P, gamma=2, w_levels=2, low_precision=3)
    b = _t(P.b)
    for prec in (xdg.XDG_PREC_F32, xdg.XDG_PREC_F64, xdg.XDG_PREC_BF16):
        x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
        info = H.solve(b, x, tol=1e-10, maxit=1000, precision=prec)
        assert info["relres"] <= 1e-10, (prec, info)
        assert _rel(_n(x), ref) < 1e-8, (prec, info)
    H.destroy()
