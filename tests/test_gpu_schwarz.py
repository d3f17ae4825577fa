"""Parity of the additive Schwarz smoother (xdg_set_schwarz; Algorithm Swz of arXiv 2003.02431,
sec. 3.3, exact patch solves, symmetric alpha^{-1/2} overlap scaling) with the CPU oracle.

* one smoothing step and the undamped preconditioner S r (through xdg_smooth from x = 0 with
  the damping set to 1) on overlapping patches with varying alpha and on the staggered
  two-partition patches: every block within 1e-10 of its own largest entry and 1e-12
  relative in the 2-norm (FP64 on both sides; a Cholesky solve against an explicit inverse)
* the damping estimate lambda_max(S M) agrees with the oracle's to 1e-10
* one cycle with Schwarz on the two finest levels: blocks within 1e-9, 2-norm 1e-11 (the patch
  inverses, explicit here and Cholesky solves in the oracle, differ by about cond(M_PP) u, and
  patches of up to 16 blocks are worse conditioned than single blocks)
* FP64 CG and the FP32-cycle flexible CG with Schwarz reach the oracle's solution within
  1e-8 relative L2, in fewer iterations than with block Jacobi; the 64^3 benchmark workload too
* distinct patch matrices are stored once (fewer inverses than patches on a Cartesian mesh)
* invalid patches are rejected with XDG_EINVAL; batch groups refuse the Schwarz smoother
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from _bounds import check_blocks  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = {
    "2d_k2": (xp.config_2d_16(max_coarse_dof=60), 2),
    "2d_k4": (xp.Config(D=2, N=13, k=4, c=(0.5, 0.5, 0), R=0.27, muA=1, muB=10, max_coarse_dof=120), 1),
    "3d_k2": (xp.Config(D=3, N=14, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000, max_coarse_dof=300), 2),
    "3d_k3": (xp.Config(D=3, N=8, k=3, c=(0.48, 0.51, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=400), 2),
}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def staggered(P, level):
    a = P.schwarz_patches(level, 0)
    b = P.schwarz_patches(level, 1)
    return np.r_[a[0], a[0][-1] + b[0][1:]], np.r_[a[1], b[1]]


def uneven(P):
    """Overlapping patches with alpha from 1 to 3 (aggregates, cut into pieces of at most
    512 / Np blocks; half of the shifted groups; pairs)."""
    a = P.aggregate_patches(1)
    b = P.schwarz_patches(1, 1)
    nb = P.nb[0]
    cap = 512 // P.Np
    keep = [i for i in range(len(b[0]) - 1) if b[1][b[0][i]] < nb // 2]
    ptr, blk = [0], []
    for p in range(len(a[0]) - 1):
        mem = list(a[1][a[0][p]:a[0][p + 1]])
        for c in range(0, len(mem), cap):
            blk += mem[c:c + cap]
            ptr.append(len(blk))
    for p in keep:
        blk += list(b[1][b[0][p]:b[0][p + 1]])
        ptr.append(len(blk))
    for i in range(0, nb // 10, 2):
        blk += [i, i + 1]
        ptr.append(len(blk))
    return np.array(ptr, np.int64), np.array(blk, np.int32)


def schwarz_levels(P):
    return [1, 2] if P.n_levels > 2 else [1]


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    cfg, gamma = CASES[request.param]
    P = xp.Problem(cfg)
    O = oracle.Hierarchy(P, gamma=gamma)
    oracle.set_w_levels(O, 2)
    G = xdg.Hierarchy.from_problem(P, gamma=gamma, w_levels=2, low_precision=1)
    for lv in schwarz_levels(P):
        patches = staggered(P, lv)
        O.set_patches(lv - 1, patches, mode=1)
        G.set_schwarz(lv, patches)
    return request.param, P, O, G


def test_damping_estimate_parity(case):
    name, P, O, G = case
    inf = G.info()
    for lv in schwarz_levels(P):
        o = O.level(lv - 1)
        assert abs(inf["lambda_max"][lv - 1] - o["lmax"]) <= 1e-10 * o["lmax"], (name, lv)
        assert abs(inf["omega"][lv - 1] - o["omega"]) <= 1e-10 * o["omega"]


def test_distinct_inverses_are_shared(case):
    name, P, O, G = case
    s = G.schwarz_info(1)
    assert s["n_patches"] == len(staggered(P, 1)[0]) - 1 and s["overlap"] == 1
    assert 1 <= s["n_distinct"] <= s["n_patches"]
    if P.D == 3 and P.cfg.N >= 14:
        assert s["n_distinct"] < s["n_patches"], s


@pytest.mark.parametrize("patch_kind", ["staggered", "uneven"])
def test_smoothing_step_parity(case, patch_kind):
    name, P, O, G = case
    if patch_kind == "uneven":
        patches = uneven(P)
        O2 = oracle.Hierarchy(P)
        O2.set_patches(0, patches, mode=1)
        G2 = xdg.Hierarchy.from_problem(P)
        G2.set_schwarz(1, patches)
        assert G2.schwarz_info(1)["overlap"] == 1
    else:
        O2, G2 = O, G
    om = O2.level(0)["omega"]
    G2.set_damping(1, om)
    rng = np.random.default_rng(7)
    b, x = rng.standard_normal(P.dof), rng.standard_normal(P.dof)
    ref = O2.smooth(0, b, x)
    out = torch.empty(P.dof, dtype=torch.float64, device=DEV)
    G2.smooth(1, _t(b), _t(x), out)
    got = _n(out)
    check_blocks(got, ref, P.Np, 1e-10, (name, patch_kind))
    assert _rel(got, ref) < 1e-12
    # from x = 0 with omega = 1: the preconditioner itself, S b
    G2.set_damping(1, 1.0)
    G2.smooth(1, _t(b), None, out)
    ref0 = O2.schwarz(0, b)
    check_blocks(_n(out), ref0, P.Np, 1e-10, (name, patch_kind, "S b"))
    G2.set_damping(1, om)


def test_cycle_parity(case):
    name, P, O, G = case
    for l in range(P.n_levels - 1):
        G.set_damping(l + 1, O.level(l)["omega"])
    rng = np.random.default_rng(8)
    for b in (P.b.reshape(-1), rng.standard_normal(P.dof)):
        ref = O.vcycle(b)
        x = torch.empty(P.dof, dtype=torch.float64, device=DEV)
        G.vcycle(_t(b), x)
        got = _n(x)
        check_blocks(got, ref, P.Np, 1e-9, name)
        assert _rel(got, ref) < 1e-11, name


def test_solves_reach_oracle_solution(case):
    name, P, O, G = case
    ref, it_o, rr, _ = O.pcg(P.b, tol=1e-14, maxit=600)
    b = _t(P.b)
    its = {}
    for prec in (xdg.XDG_PREC_F64, xdg.XDG_PREC_F32):
        x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
        info = G.solve(b, x, tol=1e-11, maxit=600, precision=prec)
        its[prec] = info["iterations"]
        assert _rel(_n(x), ref) < 1e-8, (name, prec, info)
    _, it_o11, _, _ = O.pcg(P.b, tol=1e-11, maxit=600)
    assert abs(its[xdg.XDG_PREC_F64] - it_o11) <= 2, (its, it_o11)
    # block Jacobi needs at least as many iterations
    GB = xdg.Hierarchy.from_problem(P, gamma=CASES[name][1], w_levels=2)
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    assert GB.solve(b, x, tol=1e-11, maxit=600)["iterations"] >= its[xdg.XDG_PREC_F64]


def test_back_to_block_jacobi():
    P = xp.Problem(xp.config_2d_16(max_coarse_dof=60))
    G = xdg.Hierarchy.from_problem(P, gamma=2)
    b = _t(P.b)
    x0 = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    it_bj = G.solve(b, x0, tol=1e-11)["iterations"]
    G.set_schwarz(1, staggered(P, 1))
    x1 = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    it_swz = G.solve(b, x1, tol=1e-11)["iterations"]
    G.set_schwarz(1, None)
    assert G.schwarz_info(1)["n_patches"] == 0
    x2 = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    assert G.solve(b, x2, tol=1e-11)["iterations"] == it_bj
    assert torch.equal(x0, x2)
    assert it_swz <= it_bj


def test_invalid_patches_rejected():
    P = xp.Problem(xp.config_2d_16(max_coarse_dof=60))
    G = xdg.Hierarchy.from_problem(P)
    nb = P.nb[0]
    bad = [
        (np.array([0, nb - 1], np.int64), np.arange(1, nb, dtype=np.int32)),           # block 0 uncovered
        (np.array([0, nb], np.int64), np.arange(nb, dtype=np.int32)[::-1].copy()),     # not ascending
        (np.array([0, 2, nb + 2], np.int64), np.r_[0, nb, np.arange(nb)].astype(np.int32)),  # out of range
        (np.array([0, nb], np.int64), np.arange(nb, dtype=np.int32)),                  # too many modes
    ]
    for patches in bad:
        with pytest.raises(xdg.XdgError) as e:
            G.set_schwarz(1, patches)
        assert e.value.code == xdg.XDG_EINVAL
    # the handle still solves with block Jacobi
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    assert G.solve(_t(P.b), x, tol=1e-10)["status"] == xdg.XDG_OK


@pytest.mark.slow
def test_full_size_schwarz_solves():
    """The 64^3 workload with Schwarz on the two finest levels, in the benchmark's cycle (W on
    two levels, autotuned storage and outer apply): FP32-cycle and FP64 solves within 1e-8 of
    the oracle's solution (oracle PCG with block Jacobi to 1e-13: the solution is unique)."""
    P = xp.Problem(xp.config_3d_64(max_coarse_dof=1000))
    O = oracle.Hierarchy(P, gamma=2)
    oracle.set_w_levels(O, 2)
    ref, _, rr, _ = O.pcg(P.b, tol=1e-13, maxit=400)
    O.close()
    G = xdg.Hierarchy.from_problem(P, gamma=2, w_levels=2, low_precision=3)
    for lv in (1, 2):
        G.set_schwarz(lv, staggered(P, lv))
    b = _t(P.b)
    for prec in (xdg.XDG_PREC_F32, xdg.XDG_PREC_F64):
        x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
        info = G.solve(b, x, tol=1e-10, maxit=400, precision=prec)
        assert _rel(_n(x), ref) < 1e-8, (prec, info)
    G.destroy()
