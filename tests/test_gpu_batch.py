"""Batched solve (many independent problems in one graph launch) against the CPU oracle.

Every problem of the batch is compared with the oracle's hierarchy of that problem alone:
  * level operators (Galerkin products of the union hierarchy, per problem): 1e-12 relative
  * every problem's damping (its own Lanczos estimate) against the oracle's: 1e-10 relative
  * one multigrid cycle of the union hierarchy, restricted to each problem: 1e-12 relative with
    the same damping on both sides, times max(1, cond/1e4) of the problem's coarsest matrix
    (explicit inverse vs Cholesky solve, as in the single-problem coarse-solve test)
  * the batched CG / flexible CG solution of each problem: 1e-8 relative L2 against the
    oracle's solution converged to 1e-13
  * per-problem iteration counts equal (within one) those of the same problem solved alone
Edge cases: a zero right-hand side (0 iterations, x = 0), an iteration limit that stops every
problem (ENOTCONV reported per problem), a batch of one, host vectors, and repeatability.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from conftest import dense_from_bsr  # noqa: E402
from paper_2003_02431_gb300 import xdg  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GAMMA = 2
OMEGA_FIXED = 0.5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).to(DEV)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def batch():
    # uneven sizes, all three block sizes of 2D k = 2, 3, 4, mixed diffusivity ratios
    cfgs = xp.batch_configs(11, seed=20030244, N_range=(8, 22), ks=(2, 3, 4), max_levels=4)
    probs = [xp.Problem(c) for c in cfgs]
    orc = [oracle.Hierarchy(p, gamma=GAMMA) for p in probs]
    bt = xdg.Batch(probs, gamma=GAMMA, low_precision=1)
    return probs, orc, bt


def _concat(bt, parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])


def test_groups_partition_the_batch(batch):
    probs, _, bt = batch
    inf = bt.info()
    assert inf["n_problems"] == len(probs)
    assert inf["total_dof"] == sum(p.dof for p in probs)
    seen = []
    for g in range(inf["n_groups"]):
        H, mem = bt.group(g)
        seen += mem
        assert len({probs[i].Np for i in mem}) == 1
        assert H.nb == [sum(probs[i].nb[l] for i in mem) for l in range(len(H.nb))]
        assert mem == sorted(mem)
    assert sorted(seen) == list(range(len(probs)))
    assert inf["n_groups"] == len({p.Np for p in probs})


def test_union_operators_and_cycle_match_each_problem(batch):
    probs, orc, _ = batch
    bt = xdg.Batch(probs, gamma=GAMMA, low_precision=1)  # its damping is changed below
    rng = np.random.default_rng(3)
    for g in range(bt.info()["n_groups"]):
        H, mem = bt.group(g)
        Np = H.Np
        # Galerkin operators of every level, block rows of each problem
        for l in range(len(H.nb)):
            rp, cl, vl = H.export_level(l + 1)
            b0 = 0
            for i in mem:
                lv = orc[i].level(l)
                nb = lv["nb"]
                rows = slice(b0, b0 + nb)
                sub_rp = rp[b0:b0 + nb + 1] - rp[b0]
                z0, z1 = rp[b0], rp[b0 + nb]
                assert np.array_equal(sub_rp, lv["row_ptr"]), (g, l, i)
                assert np.array_equal(cl[z0:z1] - b0, lv["col"]), (g, l, i)
                scale = np.abs(lv["val"]).max()
                assert np.abs(vl[z0:z1] - lv["val"]).max() <= 1e-12 * scale, (g, l, i)
                b0 += nb
                del rows
        # every problem's own damping: its Lanczos estimate agrees with the oracle's
        for s, i in enumerate(mem):
            for l in range(len(H.nb) - 1):
                om, lm = H.get_damping(l + 1, s)
                lv = orc[i].level(l)
                assert abs(om - lv["omega"]) <= 1e-10 * lv["omega"], (g, i, l)
                assert abs(lm - lv["lmax"]) <= 1e-10 * lv["lmax"], (g, i, l)
        # one cycle on the union = the problems' own cycles, with the same damping on both sides
        # (a cycle is as sensitive to the damping as its size; the estimates agree to 1e-10)
        for l in range(len(H.nb) - 1):
            H.set_damping(l + 1, OMEGA_FIXED)
        parts = [rng.standard_normal(probs[i].dof) for i in mem]
        r = _t(_concat(bt, parts))
        z = torch.empty_like(r)
        H.vcycle(r, z)
        zz = _n(z)
        o = 0
        for i, p in zip(mem, parts):
            Oi = oracle.Hierarchy(probs[i], gamma=GAMMA, omega=OMEGA_FIXED)
            ref = Oi.vcycle(p)
            # the coarsest solves (explicit inverse here, Cholesky in the oracle) differ by about
            # cond * eps: the bound of the single-problem coarse-solve parity test
            lc = Oi.level(probs[i].n_levels - 1)
            cond = np.linalg.cond(dense_from_bsr(lc["row_ptr"], lc["col"], lc["val"]))
            assert _rel(zz[o:o + p.size], ref) < 1e-12 * max(1.0, cond / 1e4), (g, i, cond)
            o += p.size
        assert Np in (6, 10, 15)
    bt.destroy()


@pytest.fixture(scope="module")
def reference_solutions(batch):
    probs, orc, _ = batch
    out = []
    for p, O in zip(probs, orc):
        x, it, rr, _ = O.pcg(p.b, tol=1e-13, maxit=500)
        assert rr < 1e-12
        out.append(x)
    return out


@pytest.mark.parametrize("prec", [xdg.XDG_PREC_F64, xdg.XDG_PREC_F32])
def test_batched_solve_matches_oracle(batch, reference_solutions, prec):
    probs, _, bt = batch
    b = _t(_concat(bt, [p.b for p in probs]))
    x = torch.zeros_like(b)
    res = bt.solve(b, x, tol=1e-10, maxit=300, precision=prec)
    xx = _n(x)
    off = bt.offsets
    for i, p in enumerate(probs):
        r = res["problems"][i]
        assert r["status"] == xdg.XDG_OK, (i, r)
        assert r["relres"] < 2e-10, (i, r)
        assert r["iterations"] > 0
        assert _rel(xx[off[i]:off[i + 1]], reference_solutions[i]) < 1e-8, (i, prec)
    assert res["iterations"] == max(r["iterations"] for r in res["problems"])
    assert res["launches"] > 0


def test_batched_iterations_equal_single_solves(batch):
    probs, _, bt = batch
    b = _t(_concat(bt, [p.b for p in probs]))
    x = torch.zeros_like(b)
    res = bt.solve(b, x, tol=1e-10, maxit=300)
    for i, p in enumerate(probs):
        G = xdg.Hierarchy.from_problem(p, gamma=GAMMA)
        bi, xi = _t(p.b), torch.zeros(p.dof, dtype=torch.float64, device=DEV)
        single = G.solve(bi, xi, tol=1e-10, maxit=300)
        assert abs(single["iterations"] - res["problems"][i]["iterations"]) <= 1, (i, single, res["problems"][i])
        G.destroy()


def test_batched_solve_is_repeatable_and_host_path_agrees(batch):
    probs, _, bt = batch
    bh = _concat(bt, [p.b for p in probs])
    b = _t(bh)
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    bt.solve(b, x1, tol=1e-10, precision=xdg.XDG_PREC_F32)
    bt.solve(b, x2, tol=1e-10, precision=xdg.XDG_PREC_F32)
    a1, a2 = _n(x1), _n(x2)
    assert np.array_equal(a1, a2)  # fixed-order reductions: bitwise repeatable
    xh = np.zeros_like(bh)
    rh = bt.solve_host(bh, xh, tol=1e-10, precision=xdg.XDG_PREC_F32)
    assert rh["status"] == xdg.XDG_OK
    assert np.array_equal(xh, a1)


def test_zero_rhs_and_iteration_limit(batch):
    probs, _, bt = batch
    parts = [p.b.reshape(-1).copy() for p in probs]
    parts[3][:] = 0.0
    b = _t(_concat(bt, parts))
    x = torch.zeros_like(b)
    res = bt.solve(b, x, tol=1e-10, maxit=300)
    off = bt.offsets
    assert res["problems"][3]["iterations"] == 0
    assert res["problems"][3]["status"] == xdg.XDG_OK
    assert not np.any(_n(x)[off[3]:off[4]])
    # every other problem converged regardless
    assert all(r["status"] == xdg.XDG_OK for r in res["problems"])
    x.zero_()
    res = bt.solve(b, x, tol=1e-14, maxit=2, raise_on_error=False)
    assert res["status"] == xdg.XDG_ENOTCONV
    for i, r in enumerate(res["problems"]):
        if i == 3:
            assert r["status"] == xdg.XDG_OK and r["iterations"] == 0
        else:
            assert r["status"] == xdg.XDG_ENOTCONV and r["iterations"] == 2, (i, r)


def test_batch_of_one_equals_the_single_solve():
    p = xp.Problem(xp.batch_configs(1, seed=11, N_range=(20, 20), ks=(3,), max_levels=4)[0])
    bt = xdg.Batch([p], gamma=GAMMA)
    G = xdg.Hierarchy.from_problem(p, gamma=GAMMA)
    b = _t(p.b)
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    r1 = bt.solve(b, x1, tol=1e-11)
    r2 = G.solve(b, x2, tol=1e-11)
    assert abs(r1["iterations"] - r2["iterations"]) <= 1
    assert _rel(_n(x1), _n(x2)) < 1e-9
    bt.destroy()
    G.destroy()
