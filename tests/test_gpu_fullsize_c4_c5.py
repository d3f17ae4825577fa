"""Full-size parity of the batched and learned-correction workloads, on sampled outputs.

* batched (256 2D problems, 18.8 M DOF, the benchmark's configuration: W on 2 levels, FP32
  cycle inside FP64 flexible CG): eight problems drawn with numpy PCG64(96), each against the
  oracle's own solve of that problem (PCG to 1e-12), within 1e-8 relative L2
* learned correction (trained on 48^3 problems, applied in the solve of the 64^3 problem with the
  held-out radius 0.29): the solution within 1e-8 of the oracle's
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import xdg_problem as xp  # noqa: E402
from paper_2003_02431_gb300 import learned, xdg  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_c4_batched_solve_sampled_problems():
    import bench
    probs = bench.make_batch_problems()
    assert len(probs) == 256
    bt = xdg.Batch(probs, gamma=bench.GAMMA, w_levels=bench.W_LEVELS, low_precision=1)
    bh = np.concatenate([p.b.reshape(-1) for p in probs])
    b = torch.from_numpy(bh).to(DEV)
    x = torch.zeros_like(b)
    res = bt.solve(b, x, tol=1e-11, maxit=1000, precision=xdg.XDG_PREC_F32)
    torch.cuda.synchronize()
    xx = x.cpu().numpy()
    off = bt.offsets
    assert all(r["status"] == xdg.XDG_OK for r in res["problems"])
    rng = np.random.Generator(np.random.PCG64(96))
    for i in sorted(rng.choice(256, 8, replace=False)):
        P = probs[i]
        O = oracle.Hierarchy(P, gamma=bench.GAMMA)
        oracle.set_w_levels(O, bench.W_LEVELS)
        xref, it, rr, _ = O.pcg(P.b, tol=1e-12, maxit=1000)
        assert rr < 1e-11
        assert _rel(xx[off[i]:off[i + 1]], xref) < 1e-8, (i, P.Np, P.dof)
        O.close()
    bt.destroy()


def test_c5_learned_solve_reaches_oracle_solution():
    import bench
    rng = np.random.Generator(np.random.PCG64(bench.LEARNED_SEED))
    radii = []
    while len(radii) < 2:
        r = float(rng.uniform(0.2, 0.4))
        if all(abs(r - h) > 0.005 for h in bench.HELD_OUT_RADII):
            radii.append(r)
    train = learned.SampleSet()
    for R in radii:
        P = xp.Problem(xp.config_3d_64(N=48, R=R, max_coarse_dof=1000))
        H = xdg.Hierarchy.from_problem(P, gamma=bench.GAMMA, w_levels=bench.W_LEVELS, low_precision=1)
        learned.attach_units(H, P)
        bt = torch.from_numpy(P.b.reshape(-1).copy()).to(DEV)
        train.add(H, learned.solver_residuals(H, bt, 12))
        H.destroy()
    net = learned.network_for(P, seed=bench.LEARNED_SEED)
    learned.train(net, train, epochs=30, batch=512, lr=2e-3, seed=bench.LEARNED_SEED)
    P = xp.Problem(xp.config_3d_64(R=0.29, max_coarse_dof=1000))
    H = xdg.Hierarchy.from_problem(P, gamma=bench.GAMMA, w_levels=bench.W_LEVELS, low_precision=1)
    learned.attach_units(H, P)
    H.learned_enable(net, theta=0.25)
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(DEV)
    x = torch.zeros_like(b)
    info = H.solve(b, x, tol=1e-11, maxit=1000, precision=xdg.XDG_PREC_F32)
    torch.cuda.synchronize()
    O = oracle.Hierarchy(P, gamma=bench.GAMMA)
    oracle.set_w_levels(O, bench.W_LEVELS)
    xref, it, rr, _ = O.pcg(P.b, tol=1e-12, maxit=1000)
    assert rr < 1e-11
    assert _rel(x.cpu().numpy(), xref) < 1e-8, info
