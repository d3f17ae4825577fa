"""The allocation-free restriction entry point against the oracle and the handle-based one.

xdg_restrict_noalloc serves callers that cannot call cudaMalloc (memory arenas that own all
device memory, plugins whose host forbids allocations, real-time loops). It keeps its scratch
in a fixed device array inside the library. This file checks, on two calls in a row:

* its output against the oracle's restriction of the oracle's residual,
  rc = R^T (b - M x) (Eq. XDGrestrictionMatrix / Algorithm 4's restriction step), entry by
  entry within c 2^-53 (|R|^T (|b| + |M||x|)), and against xdg_restrict (the same kernels with
  scratch that xdg_create_hierarchy allocated);
* that the second call is not affected by what the first one left in the shared array;
* that a call changes the device's free memory by nothing (after one warm-up call, which may
  load the kernels' code);
* that nb_fine*Np exactly at the scratch size is accepted and one block more is rejected
  before any work is enqueued.

It sits in a file of its own, collected last, and passes alone in a fresh process as well as
after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U = 2.0 ** -53


def _children(agg, nbc):
    order = np.argsort(agg, kind="stable")  # children of every coarse block, ascending
    ptr = np.zeros(nbc + 1, dtype=np.int64)
    np.add.at(ptr, agg + 1, 1)
    return np.cumsum(ptr), order.astype(np.int32)


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt).reshape(-1)).to(DEV)


def _abs_bsr_spmv(rp, col, val, x):
    return oracle.bsr_spmv(rp, col, np.abs(val), np.abs(x)).reshape(-1)


def _oracle_restrict(rp, col, val, agg, R, b, x, nbc):
    """Expected rc and its element-wise rounding bound (both computed on the host)."""
    r = b - oracle.bsr_spmv(rp, col, val, x).reshape(-1) if x is not None else b
    ref = oracle.restrict(agg, R, r, nbc).reshape(-1)
    mag = np.abs(b) + (_abs_bsr_spmv(rp, col, val, x) if x is not None else 0.0)
    bound = oracle.restrict(agg, np.abs(R), mag, nbc).reshape(-1)
    Np = R.shape[-1]
    row_len = int(np.max(np.diff(rp))) * Np
    # both sides round: the residual (row_len + 1 terms) and the restriction sum (children x Np)
    kids = int(np.max(np.bincount(agg, minlength=nbc)))
    return ref, 2 * (row_len + kids * Np + 4) * U * bound


def _check(out, ref, bound, what):
    o = out.cpu().numpy()
    bad = np.abs(o - ref) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(o - ref) - bound)))


@pytest.mark.parametrize("cfg", [xp.config_2d_16(max_coarse_dof=60),
                                 xp.Config(D=3, N=10, k=2, c=(0.5, 0.5, 0.5), R=0.31, muA=1, muB=1000,
                                           max_coarse_dof=300)])
def test_noalloc_restriction_matches_oracle_and_handle_path(cfg):
    P = xp.Problem(cfg)
    G = xdg.Hierarchy.from_problem(P)
    Np, nbf, nbc = P.Np, P.nb[0], P.nb[1]
    agg = np.asarray(P.agg[0])
    cptr, ch = _children(agg, nbc)
    args = dict(row_ptr=_dev(P.row_ptr, np.int64), col=_dev(P.col, np.int32), val=_dev(P.val, np.float64),
                R=_dev(P.R[0], np.float64), child_ptr=_dev(cptr, np.int64), child=_dev(ch, np.int32))
    rng = np.random.default_rng(17)
    for call in range(2):  # two calls in a row share the fixed scratch
        bh = rng.standard_normal(nbf * Np)
        xh = rng.standard_normal(nbf * Np) if call == 0 else None
        b = _dev(bh, np.float64)
        x = _dev(xh, np.float64) if xh is not None else None
        ref, bound = _oracle_restrict(P.row_ptr, P.col, P.val, agg, P.R[0], bh, xh, nbc)
        out = torch.full((nbc * Np,), np.nan, dtype=torch.float64, device=DEV)
        xdg.restrict_noalloc(Np, nbf, nbc, b=b, x=x, rc=out, **args)
        torch.cuda.synchronize()
        _check(out, ref, bound, ("oracle", call))
        handle = torch.empty(nbc * Np, dtype=torch.float64, device=DEV)
        G.restrict(1, b, x, handle)
        torch.cuda.synchronize()
        assert torch.equal(out, handle), call  # same kernels, same summation order


def _diagonal_level(nb, Np, nbc, seed):
    """A block-diagonal operator with random blocks on nb blocks, children f -> f mod nbc."""
    rng = np.random.default_rng(seed)
    rp = np.arange(nb + 1, dtype=np.int64)
    col = np.arange(nb, dtype=np.int32)
    val = rng.standard_normal((nb, Np, Np))
    R = rng.standard_normal((nb, Np, Np))
    agg = (np.arange(nb) % nbc).astype(np.int32)
    return rp, col, val, R, agg


def test_noalloc_allocates_nothing_and_accepts_the_maximum_size():
    Np = 10
    nb = xdg.NOALLOC_MAX_ENTRIES // Np  # nb_fine * Np as close to the scratch size as Np allows
    nbc = 1024
    rp, col, val, R, agg = _diagonal_level(nb, Np, nbc, 23)
    cptr, ch = _children(agg, nbc)
    rng = np.random.default_rng(29)
    bh, xh = rng.standard_normal(nb * Np), rng.standard_normal(nb * Np)
    args = dict(row_ptr=_dev(rp, np.int64), col=_dev(col, np.int32), val=_dev(val, np.float64),
                R=_dev(R, np.float64), child_ptr=_dev(cptr, np.int64), child=_dev(ch, np.int32),
                b=_dev(bh, np.float64), x=_dev(xh, np.float64))
    out = torch.full((nbc * Np,), np.nan, dtype=torch.float64, device=DEV)
    xdg.restrict_noalloc(Np, nb, nbc, rc=out, **args)  # warm-up: kernel code may load now
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out.fill_(np.nan)
    xdg.restrict_noalloc(Np, nb, nbc, rc=out, **args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref, bound = _oracle_restrict(rp, col, val, agg, R, bh, xh, nbc)
    _check(out, ref, bound, "maximum size")


def test_noalloc_rejects_sizes_beyond_the_scratch():
    Np = 10
    nbf = xdg.NOALLOC_MAX_ENTRIES // Np + 1
    nbc = 1
    # tensors of the full stated lengths, so that only the scratch limit can reject the call
    i64 = torch.zeros(nbf + 1, dtype=torch.int64, device=DEV)
    i32 = torch.zeros(nbf, dtype=torch.int32, device=DEV)
    vec = torch.zeros(nbf * Np, dtype=torch.float64, device=DEV)
    blocks = torch.zeros(nbf * Np * Np, dtype=torch.float64, device=DEV)
    cptr = torch.tensor([0, nbf], dtype=torch.int64, device=DEV)
    rc = torch.zeros(nbc * Np, dtype=torch.float64, device=DEV)
    with pytest.raises(xdg.XdgError) as e:
        xdg.restrict_noalloc(Np, nbf, nbc, i64, i32, blocks, blocks, cptr, i32, vec, None, rc)
    assert e.value.code == xdg.XDG_EINVAL


def test_noalloc_binding_rejects_short_arrays():
    Np, nbf, nbc = 10, 100, 10
    rp, col, val, R, agg = _diagonal_level(nbf, Np, nbc, 31)
    cptr, ch = _children(agg, nbc)
    good = dict(row_ptr=_dev(rp, np.int64), col=_dev(col, np.int32), val=_dev(val, np.float64),
                R=_dev(R, np.float64), child_ptr=_dev(cptr, np.int64), child=_dev(ch, np.int32),
                b=_dev(np.ones(nbf * Np), np.float64), x=None,
                rc=torch.zeros(nbc * Np, dtype=torch.float64, device=DEV))
    for name, short in (("b", good["b"][:-1]), ("R", good["R"][:-Np]), ("rc", good["rc"][:-1]),
                        ("child", good["child"][:-1]), ("val", good["val"][:-1])):
        bad = dict(good)
        bad[name] = short
        with pytest.raises(ValueError):
            xdg.restrict_noalloc(Np, nbf, nbc, **bad)
