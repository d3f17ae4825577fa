"""Full-size mixed-precision workload: 3D unit cube, 96^3 cells, sphere radius drawn from
U(0.25, 0.4) (numpy PCG64 seed 20030243, first draw), diffusivity 1:1000, k = 3 (Np = 20),
about 18 million DOF.

* the level-1 operator apply (FP64, and the FP32/BF16 stored copies within their bounds) on
  2,000 sampled block rows, against the oracle's product of those rows
* FP32 and BF16-transfer mixed solves (flexible CG, FP64 residuals) reach the oracle's FP64
  solution (oracle PCG to 1e-12) within 1e-8 relative L2, as does the plain FP64 GPU solve
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"


def c3_config():
    rng = np.random.Generator(np.random.PCG64(20030243))
    R = float(rng.uniform(0.25, 0.4))
    return xp.config_3d_64(N=96, k=3, R=R, max_coarse_dof=2048)


@pytest.fixture(scope="module")
def c3():
    P = xp.Problem(c3_config())
    G = xdg.Hierarchy.from_problem(P, gamma=2, w_levels=2, low_precision=3)
    return P, G


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_sampled_rows_apply(c3):
    P, G = c3
    rng = np.random.default_rng(96)
    x = rng.standard_normal(P.dof)
    xt = torch.from_numpy(x).to(DEV)
    rows = np.sort(rng.choice(P.nb[0], 2000, replace=False))
    # the sampled rows as a small BSR matrix over the full column range
    rp = np.zeros(len(rows) + 1, np.int64)
    cols, vals = [], []
    for k, i in enumerate(rows):
        z0, z1 = P.row_ptr[i], P.row_ptr[i + 1]
        cols.append(P.col[z0:z1])
        vals.append(P.val[z0:z1])
        rp[k + 1] = rp[k] + (z1 - z0)
    ref = oracle.bsr_spmv(rp, np.concatenate(cols), np.concatenate(vals), x).reshape(len(rows), P.Np)
    y = torch.empty_like(xt)
    for prec, tol in ((xdg.XDG_PREC_F64, 1e-12), (xdg.XDG_PREC_F32, 1e-5), (xdg.XDG_PREC_BF16, 1e-2)):
        G.apply(1, xt, y, prec=prec)
        torch.cuda.synchronize()
        got = y.cpu().numpy().reshape(-1, P.Np)[rows]
        assert _rel(got, ref) < tol, prec


def test_mixed_solves_reach_oracle_solution(c3):
    P, G = c3
    O = oracle.Hierarchy(P, gamma=2)
    oracle.set_w_levels(O, 2)
    xref, it, rr, _ = O.pcg(P.b, tol=1e-12, maxit=400)
    assert rr < 1e-11
    O.close()
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(DEV)
    its = {}
    for prec in (xdg.XDG_PREC_F32, xdg.XDG_PREC_BF16, xdg.XDG_PREC_F64):
        x = torch.zeros_like(b)
        info = G.solve(b, x, tol=1e-11, maxit=400, precision=prec)
        torch.cuda.synchronize()
        its[prec] = info["iterations"]
        assert _rel(x.cpu().numpy(), xref) < 1e-8, (prec, info)
    assert its[xdg.XDG_PREC_F32] <= 1.5 * its[xdg.XDG_PREC_F64] + 3
