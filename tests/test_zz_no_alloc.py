"""The allocation-free restriction entry point matches the handle-based one.

xdg_restrict_noalloc serves callers that cannot call cudaMalloc (memory arenas that own all
device memory, plugins whose host forbids allocations, real-time loops). It keeps its scratch
in a fixed device array inside the library; this test checks, on two calls in a row, that its
output equals xdg_restrict's (which uses scratch allocated by xdg_create_hierarchy), that the
second call is not affected by what the first one left in the shared array, and that sizes
beyond the fixed scratch are rejected before any work is enqueued.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _children(agg, nbc):
    order = np.argsort(agg, kind="stable")  # children of every coarse block, ascending
    ptr = np.zeros(nbc + 1, dtype=np.int64)
    np.add.at(ptr, agg + 1, 1)
    return np.cumsum(ptr), order.astype(np.int32)


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt).reshape(-1)).to(DEV)


@pytest.mark.parametrize("cfg", [xp.config_2d_16(max_coarse_dof=60),
                                 xp.Config(D=3, N=10, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000,
                                           max_coarse_dof=300)])
def test_noalloc_restriction_matches_handle_path(cfg):
    P = xp.Problem(cfg)
    G = xdg.Hierarchy.from_problem(P)
    Np, nbf, nbc = P.Np, P.nb[0], P.nb[1]
    cptr, ch = _children(np.asarray(P.agg[0]), nbc)
    args = dict(row_ptr=_dev(P.row_ptr, np.int64), col=_dev(P.col, np.int32), val=_dev(P.val, np.float64),
                R=_dev(P.R[0], np.float64), child_ptr=_dev(cptr, np.int64), child=_dev(ch, np.int32))
    rng = np.random.default_rng(17)
    for call in range(2):  # two calls in a row share the fixed scratch
        b = _dev(rng.standard_normal(nbf * Np), np.float64)
        x = _dev(rng.standard_normal(nbf * Np), np.float64) if call == 0 else None
        ref = torch.empty(nbc * Np, dtype=torch.float64, device=DEV)
        G.restrict(1, b, x, ref)
        out = torch.full((nbc * Np,), np.nan, dtype=torch.float64, device=DEV)
        xdg.restrict_noalloc(Np, nbf, nbc, b=b, x=x, rc=out, **args)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.linalg.norm(o - r) <= 1e-12 * np.linalg.norm(r), call


def test_noalloc_rejects_sizes_beyond_the_scratch():
    Np = 10
    nbf = xdg.NOALLOC_MAX_ENTRIES // Np + 1
    dummy_i64 = torch.zeros(2, dtype=torch.int64, device=DEV)
    dummy_i32 = torch.zeros(2, dtype=torch.int32, device=DEV)
    dummy = torch.zeros(2, dtype=torch.float64, device=DEV)
    with pytest.raises(xdg.XdgError) as e:
        xdg.restrict_noalloc(Np, nbf, 1, dummy_i64, dummy_i32, dummy, dummy, dummy_i64, dummy_i32,
                             dummy, None, dummy)
    assert e.value.code == xdg.XDG_EINVAL
