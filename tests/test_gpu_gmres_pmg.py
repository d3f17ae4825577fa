"""Flexible GMRES and the p-multigrid preconditioner (xdg_solve_gmres, xdg_pmg_setup,
xdg_pmg_apply; arXiv 2003.02431, sec. 3.3: Algorithm pMultigrid, GMRES with PMG) against the
CPU oracle.

* PMG apply: with the inner low-order solve converged to 1e-13 the GPU's PMG equals the oracle's
  (dense direct low-order solve) within 1e-9 relative, for k_lo = 1 (n_lo = 3 in 2D, 4 in 3D)
  and k_lo = 2
* GMRES + PMG and GMRES + multigrid cycle (FP64 and FP32 cycle) reach the oracle's solution within
  1e-8 relative L2; restarts (a short restart length) keep converging
* bad options are rejected
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = {
    # name: (config, n_lo values)
    "2d_k2": (xp.config_2d_16(max_coarse_dof=60), (3,)),
    "2d_k3": (xp.Config(D=2, N=20, k=3, c=(0.46, 0.53, 0), R=0.31, muA=1, muB=100, max_coarse_dof=120), (3, 6)),
    "3d_k2": (xp.Config(D=3, N=10, k=2, c=(0.47, 0.52, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=200), (4,)),
    "3d_k3": (xp.Config(D=3, N=7, k=3, c=(0.48, 0.51, 0.5), R=0.3, muA=1, muB=1000, max_coarse_dof=300), (4, 10)),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    cfg, nlos = CASES[request.param]
    P = xp.Problem(cfg)
    O = oracle.Hierarchy(P, gamma=2)
    ref, _, rr, _ = O.pcg(P.b, tol=1e-14, maxit=600)
    return request.param, P, O, ref, nlos


def test_pmg_apply_parity(case):
    name, P, O, ref, nlos = case
    r = np.random.default_rng(4).standard_normal(P.dof)
    for n_lo in nlos:
        G = xdg.Hierarchy.from_problem(P, gamma=2)
        G.pmg_setup(n_lo, inner_tol=1e-13, inner_maxit=600)
        z = torch.empty(P.dof, dtype=torch.float64, device=DEV)
        G.pmg_apply(_t(r), z)
        expect = O.pmg(0, n_lo, r)
        assert _rel(_n(z), expect) < 1e-9, (name, n_lo)


def test_gmres_pmg_solution(case):
    name, P, O, ref, nlos = case
    n_lo = nlos[0]
    G = xdg.Hierarchy.from_problem(P, gamma=2)
    G.pmg_setup(n_lo, inner_tol=1e-8, inner_maxit=400)
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve_gmres(_t(P.b), x, tol=1e-11, maxit=2000, restart=60, preconditioner=1)
    assert info["relres"] <= 1e-11
    assert _rel(_n(x), ref) < 1e-8, (name, info)


@pytest.mark.parametrize("prec", [xdg.XDG_PREC_F64, xdg.XDG_PREC_F32])
def test_gmres_cycle_solution(case, prec):
    name, P, O, ref, nlos = case
    G = xdg.Hierarchy.from_problem(P, gamma=2, low_precision=1)
    b = _t(P.b)
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info = G.solve_gmres(b, x, tol=1e-11, maxit=600, restart=40, precision=prec)
    assert _rel(_n(x), ref) < 1e-8, (name, info)
    # CG with the same cycle for comparison: GMRES minimises the residual, so it needs at most
    # about as many steps
    xc = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    it_cg = G.solve(b, xc, tol=1e-11, maxit=600, precision=prec)["iterations"]
    assert info["iterations"] <= it_cg + 5, (info["iterations"], it_cg)
    # a short restart still converges
    x2 = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    info2 = G.solve_gmres(b, x2, tol=1e-11, maxit=2000, restart=5, precision=prec)
    assert _rel(_n(x2), ref) < 1e-8 and info2["iterations"] >= info["iterations"]


def test_bad_options():
    P = xp.Problem(xp.config_2d_16(max_coarse_dof=60))
    G = xdg.Hierarchy.from_problem(P)
    x = torch.zeros(P.dof, dtype=torch.float64, device=DEV)
    with pytest.raises(xdg.XdgError):   # no p-multigrid set up yet
        G.solve_gmres(_t(P.b), x, preconditioner=1)
    with pytest.raises(xdg.XdgError):   # no FP32 copy in this hierarchy
        G.solve_gmres(_t(P.b), x, precision=xdg.XDG_PREC_F32)
    for n_lo in (0, P.Np, 5):
        with pytest.raises(xdg.XdgError):
            G.pmg_setup(n_lo)
    info = G.solve_gmres(_t(P.b), x, tol=1e-12, maxit=3, raise_on_error=False)
    assert info["status"] == xdg.XDG_ENOTCONV and info["iterations"] == 3
