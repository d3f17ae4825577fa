"""The bounded waits on the GPU: a wait that runs out reports an error status and the context
stays usable (no trap, no hang).

The fused small-level cycle separates its steps by grid-wide barriers; every barrier polls a
bounded number of times. xdg_test_barrier_timeout makes each barrier wait for one CTA more than
the launch has, so every wait runs out: the solve must return XDG_ETIMEOUT within seconds, and
the next solve, with the normal barriers, must give the same result as before.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_fused_barrier_timeout_reports_and_recovers():
    P = xp.Problem(xp.Config(D=3, N=16, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000, max_coarse_dof=300))
    H = xdg.Hierarchy.from_problem(P, gamma=2, w_levels=2, low_precision=1, fused_coarse=2)
    assert H.info()["fused_level"] > 0, "the fused small-level cycle is not in use"
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(DEV)
    x0 = torch.zeros_like(b)
    ok = H.solve(b, x0, tol=1e-10, maxit=200, precision=xdg.XDG_PREC_F32)
    assert ok["status"] == xdg.XDG_OK
    H.test_barrier_timeout(True)
    x1 = torch.zeros_like(b)
    t = time.perf_counter()
    info = H.solve(b, x1, tol=1e-10, maxit=5, precision=xdg.XDG_PREC_F32, raise_on_error=False)
    elapsed = time.perf_counter() - t
    assert info["status"] == xdg.XDG_ETIMEOUT, info
    assert elapsed < 30.0
    H.test_barrier_timeout(False)
    x2 = torch.zeros_like(b)
    again = H.solve(b, x2, tol=1e-10, maxit=200, precision=xdg.XDG_PREC_F32)
    assert again["status"] == xdg.XDG_OK and again["iterations"] == ok["iterations"]
    assert torch.equal(x0, x2)


def test_barrier_timeout_needs_a_fused_cycle():
    P = xp.Problem(xp.config_2d_16(max_coarse_dof=60))
    H = xdg.Hierarchy.from_problem(P, low_precision=1, fused_coarse=1)
    with pytest.raises(xdg.XdgError) as e:
        H.test_barrier_timeout(True)
    assert e.value.code == xdg.XDG_EINVAL
