#!/usr/bin/env python3
"""Benchmark of the multigrid-preconditioned XDG solve on GB300 (libxdg through its C ABI).

Workload (synthetic, generated in-process): 3D XDG Poisson problem on the unit cube, 64^3
Cartesian cells, spherical interface (centre (0.5,0.5,0.5), radius 0.31), diffusivity 1 inside /
1000 outside, SIP, DG degree k=2 (Np=10), agglomeration threshold 0.1, manufactured smooth
solution: 266,232 blocks, 2,662,320 DOF, 1,849,276 non-zero 10x10 blocks, 5 levels.

A step is one complete solve from x = 0 to ||b - M x|| <= 1e-10 ||b|| (the parity tests show
the solution then lies within 1e-8 relative L2 of the FP64 oracle's solution). The headline
path is flexible CG in FP64 (residuals, updates, inner products; the operator apply q = M p
FP64-accurate from FP32 pairs when the creation-time autotuner keeps it) preconditioned by an
FP32 W-cycle (block-Jacobi smoothing, fused residual-restriction, prolongation, FP64 coarsest
solve; level 1 read from its symmetric storage when kept); the plain FP64 path (CG with the
FP64 W-cycle and the FP64 apply) is timed next to it. value = DOF solved per second of the
headline path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xdg|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "XDG solve time to 1e-8 rel. L2 & V-cycle MDOF/s vs plain FP64 path, 1 GB300"
WORKLOAD = "xdg-poisson-3d-64^3-k2-sphere-R0.31-mu1:1000"
TOL = 1e-10
GAMMA, W_LEVELS = 2, 2   # W-cycle on the two finest levels, V-cycle below


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


SIZE = 64  # cells per direction (--size; the benchmark workload is 64)

# level-1 kernels timed by the bench: (full storage, symmetric storage) kernel names
KERNEL_NAMES = {
    "resid_rt_f32": ("k_resid_rt_lp<10,float,float,1,0>", "k_resid_rt_lp_sym<10,float>",
                     "level-1 FP32 residual and R^T (restriction phase 1)"),
    "smooth_f32": ("k_smooth_lp<10,float,0,0>", "k_smooth_lp_sym<10>", "level-1 FP32 block-Jacobi sweep"),
    "apply_f32": ("k_spmv_lp<10,float,float,0>", None, "level-1 FP32 operator apply"),
    "apply_f64": ("k_spmv<10,0>", None, "level-1 FP64 operator apply (the FP64 path's CG)"),
    "apply_pair": ("k_spmv_dot_df<10>", "k_spmv_dot_df_sym<10>",
                   "level-1 FP64-accurate apply from FP32 pairs (the mixed solve's flexible CG)"),
}
# the largest kernel of the mixed solve's device time (the launch list of the solve), the
# largest kernel of the cycle, and the FP64 path's apply (ALU-bound)
DOMINANT = "apply_pair"
DOMINANT_HBM = "resid_rt_f32"
DOMINANT_FP64 = "apply_f64"
PARITY_BOUND = 1e-8   # the metric's tolerance: relative L2 distance to the oracle's solution


def csrc_digest():
    """sha256 (first 16 hex digits) of the CUDA sources, to tell whether a recorded ncu
    measurement was taken on the kernels that run now."""
    import hashlib
    d = os.path.join(ROOT, "paper_2003_02431_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, alg_bytes):
    """DRAM bytes (read + write) per launch of `kernel`, from a committed ncu summary line
    `traffic_per_launch kernel=<name> size=<N> bytes=<B> alg_bytes=<A> csrc_sha256=<digest>`
    whose digest matches the current sources (else None: the counters are stale). A capture on a
    smaller mesh (the capture-size rule) is scaled to this launch by the algorithmic bytes:
    B * alg_bytes / A (the kernel streams its storage once, so its traffic grows with it)."""
    import glob
    import re
    digest = csrc_digest()
    pat = re.compile(r"traffic_per_launch kernel=(\S+) size=(\d+) bytes=(\d+) alg_bytes=(\d+) "
                     r"csrc_sha256=([0-9a-f]+)")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for m in pat.finditer(f.read()):
                if m.group(1) == kernel and m.group(5) == digest:
                    return int(round(int(m.group(3)) * float(alg_bytes) / int(m.group(4))))
    return None


# FP64 ALU peak from unit counts and clocks: 152 SMs x 2070 MHz x 4 FP64 flop per SM and clock
# (2 FMA), the rate of GB300's nominal 1.25 TFLOP/s FP64
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12


def max_over_ranks(value, dist, device=None):
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    import torch
    dev = "cpu" if dist.get_backend() == "gloo" else device
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, steps, seconds):
    """Whole-job throughput in millions of units per second: every rank processes its own
    copy of the workload (replicas), the job takes its slowest rank's time."""
    return world * units_per_rank * steps / seconds / 1e6


def make_problem():
    import xdg_problem as xp
    return xp.Problem(xp.config_3d_64(N=SIZE, max_coarse_dof=1000))


def oracle_hierarchy(P):
    import oracle
    O = oracle.Hierarchy(P, gamma=GAMMA)
    oracle.set_w_levels(O, W_LEVELS)
    return O


def oracle_solution(P, tol=1e-13):
    """The oracle's FP64 solution of M x = b: PCG to a relative residual of `tol`."""
    O = oracle_hierarchy(P)
    x, it, rr, _ = O.pcg(P.b, tol=tol, maxit=1000)
    O.close()
    return x.reshape(-1), it, rr


def rel_l2(x, ref):
    return float(np.linalg.norm(np.asarray(x).reshape(-1) - ref) / np.linalg.norm(ref))


def oracle_sample(P, iters_needed, budget_s=10.0):
    """Time the oracle's PCG iterations on this problem (bounded samples) with all host cores
    and with one thread, and extrapolate each to the full solve's iteration count."""
    import oracle
    t = time.perf_counter()
    O = oracle_hierarchy(P)
    setup = time.perf_counter() - t
    all_threads = oracle.set_threads(os.cpu_count() or 1)

    def sample(budget):
        m, spent = 1, 0.0
        while True:
            t = time.perf_counter()
            O.pcg(P.b, tol=0.0, maxit=m)
            dt = time.perf_counter() - t
            spent += dt
            if dt >= budget / 3 or spent >= budget:
                return dt / m, m
            m *= 2

    per_all, m_all = sample(budget_s)
    oracle.set_threads(1)
    per_one, m_one = sample(budget_s)
    oracle.set_threads(all_threads)
    O.close()
    return {"per_iteration_s": per_all, "sample_iterations": m_all, "setup_s": setup,
            "est_solve_s": per_all * iters_needed, "cores": all_threads,
            "single_thread": {"per_iteration_s": per_one, "sample_iterations": m_one,
                              "est_solve_s": per_one * iters_needed}}


BATCH_N = 256
BATCH_PARITY_SAMPLES = 8
BATCH_SEED = 20030244
BATCH_WORKLOAD = ("256 independent 2D XDG Poisson problems: N~U{32..128}^2, k~U{2,3,4}, circle centre "
                  "U(0.3,0.7)^2, R~U(0.1,0.3), mu ratio 10^U(0,3), 6 aggregation levels, seed %d" % BATCH_SEED)


def make_batch_problems(n=BATCH_N):
    """The batched workload, generated on all host cores (one thread per problem)."""
    import dataclasses
    from concurrent.futures import ThreadPoolExecutor

    import xdg_problem as xp
    cfgs = [dataclasses.replace(c, nthreads=1) for c in xp.batch_configs(n, seed=BATCH_SEED)]
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        return list(ex.map(xp.Problem, cfgs))


def batched_section(xdg, torch, dev, stream, steps, warmup):
    """One step = one batched solve of all problems (a single graph launch) to TOL."""
    t = time.perf_counter()
    probs = make_batch_problems()
    gen_s = time.perf_counter() - t
    t = time.perf_counter()
    bt = xdg.Batch(probs, gamma=GAMMA, w_levels=W_LEVELS, low_precision=1, stream=stream)
    setup_s = time.perf_counter() - t
    binfo = bt.info()
    n = bt.total_dof
    bh = np.concatenate([p.b.reshape(-1) for p in probs])
    b = torch.from_numpy(bh).to(dev)
    x = torch.zeros_like(b)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(prec):
        for _ in range(warmup):
            x.zero_()
            bt.solve(b, x, tol=TOL, maxit=1000, precision=prec)
        torch.cuda.synchronize()
        res = []
        ev0.record(stream)
        for _ in range(steps):
            x.zero_()
            res.append(bt.solve(b, x, tol=TOL, maxit=1000, precision=prec))
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps, res[-1], sum(r["launches"] for r in res), x.cpu().numpy()

    ms32, r32, launches, x32 = run(xdg.XDG_PREC_F32)
    ms64, r64, _, x64 = run(xdg.XDG_PREC_F64)
    # parity of sampled problems: the oracle's solution of each, against both timed solves
    offs = np.concatenate([[0], np.cumsum([p.dof for p in probs])])
    sample = sorted(np.random.default_rng(BATCH_SEED).choice(len(probs), BATCH_PARITY_SAMPLES, replace=False))
    errs = {"mixed_f32": [], "plain_f64": []}
    for i in sample:
        ref = oracle_solution(probs[i])[0]
        for key, xs in (("mixed_f32", x32), ("plain_f64", x64)):
            errs[key].append(rel_l2(xs[offs[i]:offs[i + 1]], ref))
    its = [p["iterations"] for p in r32["problems"]]
    # end to end: host vectors in pinned memory, copies inside the call
    bp = torch.from_numpy(bh).pin_memory().numpy()
    xp_ = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    bt.solve_host(bp, xp_, tol=TOL, maxit=1000, precision=xdg.XDG_PREC_F32)
    t = time.perf_counter()
    for _ in range(steps):
        bt.solve_host(bp, xp_, tol=TOL, maxit=1000, precision=xdg.XDG_PREC_F32)
    e2e_s = (time.perf_counter() - t) / steps
    out = {
        "workload": BATCH_WORKLOAD, "problems": len(probs), "dof": n, "groups": binfo["n_groups"],
        "graph_launches_per_solve": 1,
        "mixed_f32": {"solve_ms": ms32, "mdofs": n / ms32 / 1e3, "iterations_min_median_max":
                      [min(its), int(np.median(its)), max(its)], "max_relres": r32["relres"]},
        "plain_f64": {"solve_ms": ms64, "mdofs": n / ms64 / 1e3, "iterations_max": r64["iterations"],
                      "max_relres": r64["relres"]},
        "speedup_mixed_vs_f64": ms64 / ms32,
        "parity": {"problems": [int(i) for i in sample], "bound": PARITY_BOUND,
                   "max_rel_l2_vs_oracle": {k: max(v) for k, v in errs.items()}},
        "e2e": {"value": n / e2e_s / 1e6, "unit": "MDOF/s", "h2d_bytes_per_step": n * 8,
                "d2h_bytes_per_step": n * 8},
        "kernel_nodes_per_solve": launches / steps,
        "generate_s": gen_s, "setup_s": setup_s, "device_gb": binfo["device_bytes"] / 1e9,
        "groups_tuned": [],
    }
    # what the creation-time autotuner chose for every group (union hierarchy of one Np and depth)
    for g in range(binfo["n_groups"]):
        Hg, members = bt.group(g)
        gi = Hg.info()
        out["groups_tuned"].append({"Np": gi["Np"], "problems": len(members), "blocks_per_level": gi["nb"],
                                    "split_rows_levels": gi["split"], "outer_apply_pair": gi["outer_pair"],
                                    "symmetric_cycle": gi["symmetric_cycle"], "fused_level": gi["fused_level"]})
    bt.destroy()
    return out


LEARNED_SEED = 20030245
HELD_OUT_RADII = (0.23, 0.29, 0.37)


def learned_section(xdg, torch, dev, stream, n_train=4, budget=0.0):
    """Learned cut-cell correction: trained on the GPU on 48^3 k=2 sphere problems with radii
    from U(0.2, 0.4) (held-out radii excluded with a 0.005 margin), evaluated on 64^3 k=2 with
    the held-out radius 0.29: local energy gain and flexible-CG solves with and without it."""
    import xdg_problem as xp
    from paper_2003_02431_gb300 import learned
    rng = np.random.Generator(np.random.PCG64(LEARNED_SEED))
    radii = []
    while len(radii) < n_train:
        r = float(rng.uniform(0.2, 0.4))
        if all(abs(r - h) > 0.005 for h in HELD_OUT_RADII):
            radii.append(r)
    t0 = time.perf_counter()
    train = learned.SampleSet()
    for R in radii:
        P = xp.Problem(xp.config_3d_64(N=48, R=R, max_coarse_dof=1000))
        H = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=W_LEVELS, low_precision=1, stream=stream)
        learned.attach_units(H, P)
        b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
        train.add(H, learned.solver_residuals(H, b, 16))
        H.destroy()
    data_s = time.perf_counter() - t0
    net = learned.network_for(P, seed=LEARNED_SEED, stream=stream)
    n_samples = int(train.tensors()[0].shape[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = learned.train(net, train, epochs=60, batch=512, lr=2e-3, seed=LEARNED_SEED)
    train_s = time.perf_counter() - t0
    # held-out evaluation at 64^3
    P = xp.Problem(xp.config_3d_64(R=0.29, max_coarse_dof=1000))
    H = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=W_LEVELS, low_precision=1, stream=stream)
    learned.attach_units(H, P)
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
    held = learned.SampleSet()
    held.add(H, learned.solver_residuals(H, b, 8))
    Xh, uid, M, R, C = held.tensors()
    Md, Rd, Cd = M[uid.long()].double(), R.double(), C.double()
    bj = float(((torch.einsum("si,sij,sj->s", Rd, Md, Rd) - 2 * (Rd * Rd).sum(1)) / Cd).mean())
    loss = learned.evaluate(net, held)
    out = {"train": {"problems": "48^3 k=2, R from U(0.2,0.4) seed %d: %s" % (LEARNED_SEED, [round(r, 4) for r in radii]),
                     "samples": n_samples, "epochs": len(hist), "loss_first_epoch": float(hist[0]),
                     "loss_last_epoch": float(hist[-1]), "train_s": train_s, "data_s": data_s},
           "held_out": {"problem": "64^3 k=2 R=0.29", "units": int(H.n_units), "loss": loss,
                        "block_jacobi_step_loss": bj,
                        "meaning": "-1 = exact local solve of the cut-cell pair, 0 = no energy gain"}}
    x0 = torch.zeros_like(b)
    for tag, on in (("plain", False), ("learned", True)):
        if on:
            H.learned_enable(net, theta=0.25)
        x0.zero_()
        H.solve(b, x0, tol=TOL, precision=xdg.XDG_PREC_F32, time_budget_ms=budget)
        x0.zero_()
        torch.cuda.synchronize()
        # XDG_BENCH_PROFILE_RANGE=learned marks the timed learned solve for `ncu --profile-from-start off`
        prof = on and os.environ.get("XDG_BENCH_PROFILE_RANGE") == "learned"
        if prof:
            torch.cuda.profiler.start()
        info = H.solve(b, x0, tol=TOL, precision=xdg.XDG_PREC_F32, time_budget_ms=budget)
        if prof:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        out["solve_" + tag] = {"iterations": info["iterations"], "ms": info["ms"], "relres": info["relres"]}
        if tag == "plain":
            xplain = x0.clone()
    out["solution_diff_rel_l2"] = float(torch.linalg.norm(x0 - xplain) / torch.linalg.norm(xplain))
    xref = oracle_solution(P)[0]
    out["rel_l2_vs_oracle"] = {"plain": rel_l2(xplain.cpu().numpy(), xref), "learned": rel_l2(x0.cpu().numpy(), xref)}
    H.learned_enable(None)
    # the plain FP64 path on the same problem (CG with the FP64 cycle)
    x0.zero_()
    H.solve(b, x0, tol=TOL, precision=xdg.XDG_PREC_F64)
    x0.zero_()
    info = H.solve(b, x0, tol=TOL, precision=xdg.XDG_PREC_F64)
    out["solve_plain_f64"] = {"iterations": info["iterations"], "ms": info["ms"], "relres": info["relres"]}
    out["speedup_learned_vs_plain_f64"] = info["ms"] / out["solve_learned"]["ms"]
    H.destroy()
    net.destroy()
    return out


C3_SEED = 20030243
C3_STEPS = 3


def c3_config():
    """Mixed-precision workload: 96^3, sphere radius = first draw of U(0.25, 0.4) from numpy
    PCG64(20030243), mu 1:1000, k = 3 (Np = 20), about 18 million DOF."""
    import xdg_problem as xp
    rng = np.random.Generator(np.random.PCG64(C3_SEED))
    R = float(rng.uniform(0.25, 0.4))
    return xp.config_3d_64(N=96, k=3, R=R, max_coarse_dof=2048), R


def staggered_patches(P, level):
    """Schwarz patches of a level: the 2-cells-per-direction groups of its mesh and the same
    groups shifted by one cell (every block in two patches)."""
    a = P.schwarz_patches(level, 0)
    b = P.schwarz_patches(level, 1)
    return np.r_[a[0], a[0][-1] + b[0][1:]], np.r_[a[1], b[1]]


def c3_section(xdg, torch, dev, stream, P, R, gen_s, steps, with_oracle, with_schwarz=True):
    """C3 (96^3, k = 3): FP32-cycle, BF16-transfer and FP64 solves to TOL (one warm-up, `steps`
    timed solves each), the FP32-cycle solve with the additive Schwarz smoother on levels 1-2
    (timed on its second run), the level-1 pair apply against the HBM roofline. The
    solutions are compared with the FP64 GPU solve, and with the oracle's when asked (the
    oracle's solve at this size takes minutes on the host cores)."""
    n = P.dof
    t = time.perf_counter()
    H = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=W_LEVELS, low_precision=3, stream=stream)
    setup_s = time.perf_counter() - t
    hinfo = H.info()
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "xdg-poisson-3d-96^3-k3-sphere-R%.4f-mu1:1000 (seed %d)" % (R, C3_SEED), "dof": n,
           "blocks": P.nb[0], "nnz_blocks": int(P.row_ptr[-1]), "Np": P.Np, "levels": hinfo["nb"],
           "generate_s": gen_s, "setup_s": setup_s, "device_gb": hinfo["device_bytes"] / 1e9, "paths": {}}
    sols = {}
    for key, prec in (("mixed_f32", xdg.XDG_PREC_F32), ("mixed_bf16_transfers", xdg.XDG_PREC_BF16),
                      ("plain_f64", xdg.XDG_PREC_F64)):
        x.zero_()
        H.solve(b, x, tol=TOL, maxit=1000, precision=prec)
        torch.cuda.synchronize()
        its = []
        ev0.record(stream)
        for _ in range(steps):
            x.zero_()
            its.append(H.solve(b, x, tol=TOL, maxit=1000, precision=prec)["iterations"])
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        sols[key] = x.cpu().numpy()
        out["paths"][key] = {"solve_ms": ms, "iterations": its, "mdofs": n / ms / 1e3}
    for key in ("mixed_f32", "mixed_bf16_transfers"):
        out["paths"][key]["rel_l2_vs_fp64_gpu"] = rel_l2(sols[key], sols["plain_f64"])
    out["speedup_mixed_vs_f64"] = out["paths"]["plain_f64"]["solve_ms"] / out["paths"]["mixed_f32"]["solve_ms"]
    if with_schwarz:
        # the additive Schwarz smoother (staggered 2^3-cell patches, alpha = 2) on levels 1-2
        # instead of block Jacobi, the same FP32-cycle flexible CG
        t = time.perf_counter()
        for lv in (1, 2):
            H.set_schwarz(lv, staggered_patches(P, lv))
        swz_setup = time.perf_counter() - t
        x.zero_()
        H.solve(b, x, tol=TOL, maxit=1000, precision=xdg.XDG_PREC_F32)
        torch.cuda.synchronize()
        x.zero_()
        info = H.solve(b, x, tol=TOL, maxit=1000, precision=xdg.XDG_PREC_F32)
        sols["schwarz_mixed_f32"] = x.cpu().numpy()
        out["paths"]["schwarz_mixed_f32"] = {
            "solve_ms": info["ms"], "iterations": [info["iterations"]], "mdofs": n / info["ms"] / 1e3,
            "setup_s": swz_setup, "rel_l2_vs_fp64_gpu": rel_l2(sols["schwarz_mixed_f32"], sols["plain_f64"]),
            "levels": {lv: {k: H.schwarz_info(lv)[k] for k in ("n_patches", "n_distinct", "max_dof")} for lv in (1, 2)},
            "device_gb": H.info()["device_bytes"] / 1e9}
    if with_oracle:
        xref = oracle_solution(P, tol=1e-12)[0]
        for key in sols:
            out["paths"][key]["rel_l2_vs_oracle"] = rel_l2(sols[key], xref)
    hbm, hbm_kind = hbm_peak()
    if hinfo["outer_pair"]:
        ms, by = H.kernel_time(H.KERNEL_APPLY, 1, xdg.XDG_PREC_F64_PAIR, reps=10)
        name = "k_spmv_dot_df_sym<20>" if hinfo["symmetric_pair"] else "k_spmv_dot_df<20>"
    else:
        ms, by = H.kernel_time(H.KERNEL_APPLY, 1, xdg.XDG_PREC_F32, reps=10)
        name = "k_spmv_lp<20,float,float,0>"
    ach = by / (ms / 1e3) / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": name + ": level-1 outer apply of the mixed solve", "achieved": ach,
                       "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_kind": hbm_kind, "bytes": by, "ms": ms,
                       "traffic": profiled_traffic(name, by)}
    H.destroy()
    return out


def schwarz_section(xdg, torch, dev, stream, P, xref, steps, warmup):
    """The 64^3 workload with the additive Schwarz smoother (Algorithm Swz, exact patch solves) on
    the two finest levels, patches = the staggered 2^3-cell groups of each level (every block in
    two patches): FP32-cycle flexible-CG and FP64 CG solves, iterations and time, against the
    oracle's solution."""
    t = time.perf_counter()
    H = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=W_LEVELS, low_precision=1, stream=stream)
    for lv in (1, 2):
        H.set_schwarz(lv, staggered_patches(P, lv))
    setup_s = time.perf_counter() - t
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
    x = torch.zeros(P.dof, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"patches": "levels 1-2: 2-cell groups per direction and the same shifted by one cell (alpha = 2)",
           "setup_s": setup_s, "levels": {}}
    for lv in (1, 2):
        si = H.schwarz_info(lv)
        out["levels"][lv] = {"patches": si["n_patches"], "distinct_inverses": si["n_distinct"],
                             "max_dof": si["max_dof"], "device_mb": si["device_bytes"] / 1e6,
                             "omega": H.info()["omega"][lv - 1]}
    for key, prec in (("mixed_f32", xdg.XDG_PREC_F32), ("plain_f64", xdg.XDG_PREC_F64)):
        for _ in range(warmup):
            x.zero_()
            H.solve(b, x, tol=TOL, maxit=1000, precision=prec)
        torch.cuda.synchronize()
        its = []
        ev0.record(stream)
        for _ in range(steps):
            x.zero_()
            its.append(H.solve(b, x, tol=TOL, maxit=1000, precision=prec)["iterations"])
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        out[key] = {"solve_ms": ms, "iterations": its, "mdofs": P.dof / ms / 1e3,
                    "rel_l2_vs_oracle": rel_l2(x.cpu().numpy(), xref)}
    z = torch.empty_like(x)
    for _ in range(3):
        H.cycle(xdg.XDG_PREC_F32, b, z)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(20):
        H.cycle(xdg.XDG_PREC_F32, b, z)
    ev1.record(stream)
    torch.cuda.synchronize()
    out["cycle_f32_ms"] = ev0.elapsed_time(ev1) / 20
    H.destroy()
    return out


TWIN_CASES = ((2, 16), (2, 32), (2, 64), (3, 16), (3, 32), (5, 8), (5, 16), (5, 24))
# p-multigrid low orders per k (sec. 4 uses k_lo = 1 and 3) -> low-order modes in 3D
PMG_KLO = {2: (1,), 3: (1,), 5: (1, 3)}
N_LO_3D = {1: 4, 2: 10, 3: 20}


def paper_dof_table():
    """(k, N) -> DOF of the performance study's table (tab:DOFs), from the committed fixture."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "dof_table.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, N, dof = (int(v) for v in line.split())
                out[(k, N)] = dof
    return out


TOL_RESMIN = 1e-12  # residual-minimising solvers (GMRES, OrthoMG): cond(M) amplifies the residual
# the performance-study problem (f = 1, g_D = 0): its FP64 residual stalls near 1e-11 relative
# while the solution already agrees with the FP64 CG's to ~1e-13, so the residual-minimising
# solvers stop at CG's tolerance there
TWIN_TOL_RESMIN = 1e-10
TWIN_PMG_N = {2: 16, 3: 16, 5: 8}   # mesh of each k on which GMRES with p-multigrid runs
# step cap of GMRES with p-multigrid per (k, k_lo): k_lo = 1 leaves 52 of 56 modes to the block
# inverses at k = 5 and barely converges there (5e-4 after 1000 steps at N = 8)
TWIN_PMG_MAXIT = {(2, 1): 1500, (3, 1): 2500, (5, 1): 300, (5, 3): 3000}
                    # into the error, 1e-12 keeps them inside the 1e-8 error bound


def twin_section(xdg, torch, dev, stream, problems):
    """The performance study's problem (sec. 4): (-1,1)^3, sphere R = 0.7, mu 1:1000, f = 1,
    g_D = 0, k = 2, 3 and 5 on N^3 meshes. Per mesh: the DOF count against the paper's table and
    flexible CG with the FP32 W-cycle (block Jacobi; this library's headline solver) to TOL -- for
    k = 5 (Np = 56, FP64 kernels only) CG with the FP64 W-cycle. On the smallest meshes also the
    paper's other solvers, to TWIN_TOL_RESMIN: the orthonormalisation multigrid (Algorithm
    OrthoMG) with additive Schwarz smoothing (FP32 patch inverses) on every level and two passes
    per coarse visit (k = 2, 3 at N = 16), and flexible GMRES preconditioned by p-multigrid
    (Algorithm pMultigrid, the low-order system solved to 1e-5 by this library's CG) with
    k_lo = 1 (k = 2, 3 at N = 16) and k_lo = 1, 3 (k = 5 at N = 8). Graph-recorded solves are timed
    on their second run, GMRES with p-multigrid (launched step by step) on its first. Solutions
    compared with the plain FP64 GPU CG solve (to 1e-13)."""
    table = paper_dof_table()
    out = {"problem": "(-1,1)^3, sphere R=0.7, mu 1:1000, f=1, g_D=0, alpha=0.1", "tol_resmin": TWIN_TOL_RESMIN,
           "cases": []}
    for (k, N), P in problems:
        lp = P.Np <= 32
        e = {"k": k, "N": N, "Np": P.Np, "dof": P.dof, "dof_paper_table": table.get((k, N)),
             "dof_matches_table": P.dof == table.get((k, N)), "levels": len(P.nb)}
        H = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=W_LEVELS, low_precision=1 if lp else 0,
                                       stream=stream)
        b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
        x = torch.zeros(P.dof, dtype=torch.float64, device=dev)
        H.solve(b, x, tol=1e-13, maxit=3000, precision=xdg.XDG_PREC_F64)
        xref = x.cpu().numpy()

        def run(tag, fn, reps=2):
            for rep in range(reps):
                x.zero_()
                torch.cuda.synchronize()
                info = fn()
            e[tag] = {"iterations": info["iterations"], "ms": info["ms"], "relres": info["relres"],
                      "converged": info["status"] == xdg.XDG_OK,
                      "rel_l2_vs_fp64_cg": rel_l2(x.cpu().numpy(), xref)}

        if lp:
            run("cg_f32_wcycle", lambda: H.solve(b, x, tol=TOL, maxit=2000, precision=xdg.XDG_PREC_F32))
        else:
            run("cg_f64_wcycle", lambda: H.solve(b, x, tol=TOL, maxit=2000, precision=xdg.XDG_PREC_F64))
        if lp and N == 16:
            HO = xdg.Hierarchy.from_problem(P, stream=stream)
            for lv in range(1, len(P.nb)):
                HO.set_schwarz(lv, staggered_patches(P, lv))
            run("orthomg_schwarz", lambda: HO.solve_orthomg(b, x, tol=TWIN_TOL_RESMIN, maxit=600, restart=60,
                                                            coarse_passes=2, smoother_precision=xdg.XDG_PREC_F32,
                                                            raise_on_error=False))
            HO.destroy()
        if N == TWIN_PMG_N.get(k):
            for klo in PMG_KLO[k]:
                H.pmg_setup(N_LO_3D[klo], inner_tol=1e-5, inner_maxit=500)
                run("gmres_pmg_klo%d" % klo, lambda: H.solve_gmres(b, x, tol=TWIN_TOL_RESMIN,
                                                                    maxit=TWIN_PMG_MAXIT[(k, klo)], restart=60,
                                                                    preconditioner=1, raise_on_error=False), reps=1)
        H.destroy()
        out["cases"].append(e)
    return out


def solvers_section(xdg, torch, dev, stream, P, xref):
    """The 64^3 workload with the paper's other solvers, each from x = 0 to TOL_RESMIN, timed on
    its second run (GMRES with p-multigrid, launched step by step, on its first): flexible GMRES
    with the FP32 W-cycle, flexible GMRES with p-multigrid
    (Algorithm pMultigrid, k_lo = 1, the low-order system solved to 1e-5 by this library's CG),
    and the orthonormalisation multigrid (Algorithm OrthoMG with residual minimisation) with
    additive Schwarz smoothing (FP32 patch inverses) on every level. Against the oracle's
    solution."""
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
    x = torch.zeros(P.dof, dtype=torch.float64, device=dev)
    out = {"tol": TOL_RESMIN}

    def run(tag, fn, reps=2, **extra):
        for rep in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            info = fn()
        out[tag] = dict({"iterations": info["iterations"], "ms": info["ms"], "relres": info["relres"],
                         "converged": info["status"] == xdg.XDG_OK, "mdofs": P.dof / info["ms"] / 1e3,
                         "rel_l2_vs_oracle": rel_l2(x.cpu().numpy(), xref)}, **extra)

    H = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=W_LEVELS, low_precision=1, stream=stream)
    run("gmres_f32_wcycle", lambda: H.solve_gmres(b, x, tol=TOL_RESMIN, maxit=1000, restart=60,
                                                  precision=xdg.XDG_PREC_F32, raise_on_error=False), restart=60)
    H.pmg_setup(4, inner_tol=1e-5, inner_maxit=500)
    run("gmres_pmg_klo1", lambda: H.solve_gmres(b, x, tol=TOL_RESMIN, maxit=800, restart=60, preconditioner=1,
                                                raise_on_error=False), reps=1,
        restart=60, inner="CG with the W-cycle on the low-order hierarchy to 1e-5")
    H.destroy()
    HO = xdg.Hierarchy.from_problem(P, stream=stream)
    for lv in range(1, len(P.nb)):
        HO.set_schwarz(lv, staggered_patches(P, lv))
    run("orthomg_schwarz", lambda: HO.solve_orthomg(b, x, tol=TOL_RESMIN, maxit=1500, restart=60, coarse_passes=2,
                                                    smoother_precision=xdg.XDG_PREC_F32, raise_on_error=False),
        restart=60, coarse_passes=2)
    HO.destroy()
    return out


def reference_arm(args):
    """The oracle (plain FP64 CPU code) on the same workload: each step is a bounded sample of
    5 PCG iterations, extrapolated with the iteration count of the oracle's full solve."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    P = make_problem()
    O = oracle_hierarchy(P)
    _, iters, _, _ = O.pcg(P.b, tol=TOL, maxit=1000)  # warm-up: the full solve gives the count
    per = []
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        O.pcg(P.b, tol=0.0, maxit=5)
        if s >= args.warmup:
            per.append((time.perf_counter() - t) / 5)
    t_solve = statistics.mean(per) * iters
    value = P.dof / t_solve / 1e6
    # n_gpus: the launch's N (comparisons pair the two arms by it); the oracle itself runs on host cores.
    # ms_per_step is the measured time of one step (the 5-iteration sample, so that steps x
    # ms_per_step is the timed wall time); value extrapolates the sample to the full solve.
    line = {"metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": args.gpus, "device": "host CPU cores",
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(per) * 5 * 1e3,
            "step": "5 FP64 PCG iterations of the oracle's solve of the workload",
            "extrapolated_solve_ms": t_solve * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "dof": P.dof, "tol": TOL, "iterations": iters,
                       "cycle": "W(1,1) on 2 levels, block Jacobi", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "5 PCG iterations per step, extrapolated to the %d iterations "
                                       "of the oracle's full solve" % iters},
            "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xdg", choices=["xdg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 256-problem workload")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-correction section")
    ap.add_argument("--no-schwarz", action="store_true", help="skip the additive Schwarz section")
    ap.add_argument("--no-c3", action="store_true", help="skip the 96^3 k=3 mixed-precision workload")
    ap.add_argument("--no-twin", action="store_true", help="skip the performance-study problem (sec. 4)")
    ap.add_argument("--no-solvers", action="store_true", help="skip OrthoMG / GMRES / p-multigrid at 64^3")
    ap.add_argument("--c3-oracle", action="store_true",
                    help="also compare the 96^3 solutions with the oracle's (minutes of host time)")
    ap.add_argument("--fused-coarse", type=int, default=0, choices=[0, 1, 2],
                    help="small levels of the FP32 cycle as one launch: 0 autotuned, 1 never, 2 always "
                         "(for profiler runs, where the autotuner's timings are distorted)")
    ap.add_argument("--split-mask", type=int, default=-1,
                    help="force the split-row mapping per level (bit l: level l+1) instead of the autotuned one "
                         "(for profiler runs, where the autotuner's timings are distorted)")
    ap.add_argument("--outer-apply", type=int, default=0, choices=[0, 1, 2],
                    help="operator apply of the outer flexible CG: 0 autotuned, 1 FP64, 2 FP32 pairs")
    ap.add_argument("--symmetric", type=int, default=0, choices=[0, 1, 2],
                    help="symmetric storage of level 1: 0 autotuned, 1 never, 2 always")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the solve's iterations from the host (one graph launch per iteration) instead "
                         "of the device-side loop; same kernels and arithmetic, for profilers that cannot list "
                         "the kernels of a graph with conditional nodes")
    ap.add_argument("--size", type=int, default=64,
                    help="cells per direction; 64 is the benchmark workload, smaller sizes serve profiling")
    args = ap.parse_args()
    global SIZE, WORKLOAD
    SIZE = args.size
    if SIZE != 64:
        WORKLOAD = WORKLOAD.replace("64^3", "%d^3" % SIZE)
    if args.impl == "reference":
        return reference_arm(args)

    import torch

    from paper_2003_02431_gb300 import xdg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)   # the handle's stream: events are recorded on it
    warmup = max(args.warmup, 3)

    P = make_problem()
    n, Np, nb, nnzb = P.dof, P.Np, P.nb[0], int(P.row_ptr[-1])
    # the oracle's solution of the same system (host cores, outside every timed region): every
    # timed path's last solution is compared with it
    t = time.perf_counter()
    xref, it_ref, rr_ref = oracle_solution(P)
    oracle_s = time.perf_counter() - t
    # the C3 workload is generated on the host cores while the GPU works on this one (the
    # generator's ctypes call releases the GIL)
    c3 = {}
    c3_thread = None
    if not args.no_c3:
        import xdg_problem as xp

        def gen_c3():
            t0 = time.perf_counter()
            cfg, R = c3_config()
            c3["P"], c3["R"] = xp.Problem(cfg), R
            c3["gen_s"] = time.perf_counter() - t0
            if not args.no_twin:
                c3["twin"] = [((k, N), xp.Problem(xp.config_paper_twin(N=N, k=k, max_coarse_dof=1000)))
                              for k, N in TWIN_CASES]

        c3_thread = threading.Thread(target=gen_c3, daemon=True)
        c3_thread.start()
    t = time.perf_counter()
    H = xdg.Hierarchy.from_problem(P, gamma=GAMMA, w_levels=W_LEVELS, low_precision=3, stream=stream,
                                   fused_coarse=args.fused_coarse, outer_apply=args.outer_apply,
                                   symmetric=args.symmetric)
    setup_s = time.perf_counter() - t
    if args.split_mask >= 0:
        for l in range(len(P.nb)):
            H.set_split(l + 1, (args.split_mask >> l) & 1)
    hinfo = H.info()
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # a time budget (never reached) selects the host-driven iteration loop
    budget = 1e9 if args.host_loop else 0.0

    def timed_solves(prec, steps, prof=False):
        for _ in range(warmup):
            x.zero_()
            H.solve(b, x, tol=TOL, maxit=1000, precision=prec, time_budget_ms=budget)
        launches, iters = 0, []
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if prof:
            torch.cuda.profiler.start()
        ev0.record(stream)
        for _ in range(steps):
            x.zero_()
            info = H.solve(b, x, tol=TOL, maxit=1000, precision=prec, time_budget_ms=budget)
            launches += info["launches"]
            iters.append(info["iterations"])
        ev1.record(stream)
        torch.cuda.synchronize()
        if prof:
            torch.cuda.profiler.stop()
        if dist:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        if dist:
            ms = max_over_ranks(ms, dist, dev)
        return ms, launches, iters, rel_l2(x.cpu().numpy(), xref)

    # XDG_BENCH_PROFILE_RANGE=1 marks the headline timed region for `ncu --profile-from-start off`
    prof = os.environ.get("XDG_BENCH_PROFILE_RANGE") == "1"
    with ClockSampler(local) as clocks:
        t_ms, launches, iters, err32 = timed_solves(xdg.XDG_PREC_F32, args.steps, prof=prof)
    value = job_throughput(world, n, args.steps, t_ms / 1e3)
    t64_ms, _, iters64, err64 = timed_solves(xdg.XDG_PREC_F64, args.steps)
    tbf_ms, _, itersbf, errbf = timed_solves(xdg.XDG_PREC_BF16, args.steps)

    def time_call(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    z = torch.empty_like(x)
    cyc_ms = {p: time_call(lambda: H.cycle(p, b, z)) for p in (0, 1, 2)}

    # level-1 kernels of the path: mean launch duration (CUDA events on the handle's stream,
    # recorded by the library around repeated launches) and algorithmic bytes per launch
    fp64_peak = xdg.fma_peak(xdg.XDG_PREC_F64)
    hbm, hbm_kind = hbm_peak()
    kernels = {}
    for key, which, prec in (("resid_rt_f32", H.KERNEL_RESTRICT, xdg.XDG_PREC_F32),
                             ("smooth_f32", H.KERNEL_SMOOTH, xdg.XDG_PREC_F32),
                             ("apply_f32", H.KERNEL_APPLY, xdg.XDG_PREC_F32),
                             ("apply_f64", H.KERNEL_APPLY, xdg.XDG_PREC_F64),
                             ("apply_pair", H.KERNEL_APPLY, xdg.XDG_PREC_F64_PAIR)):
        if key == "apply_pair" and args.outer_apply == 1:
            continue  # no pair copy
        ms, by = H.kernel_time(which, 1, prec, reps=20)
        full, symk, what = KERNEL_NAMES[key]
        use_sym = symk is not None and (hinfo["symmetric_pair"] if key == "apply_pair" else hinfo["symmetric_cycle"])
        name = symk if use_sym else full
        kernels[key] = {"kernel": "%s: %s" % (name, what), "name": name, "ms": ms, "bytes": by,
                        "achieved_gbs": by / (ms / 1e3) / 1e9, "frac_hbm": by / (ms / 1e3) / 1e9 / hbm,
                        "storage": "symmetric (diagonal and right blocks)" if use_sym else "full"}
    flops_apply = 2.0 * nnzb * Np * Np
    ach64 = flops_apply / (kernels["apply_f64"]["ms"] / 1e3) / 1e12
    kernels["apply_f64"].update({"bound": "alu", "tflops": ach64, "frac_fp64_peak": ach64 / fp64_peak})
    # the headline's largest kernel: the pair apply when the solve uses it, else the FP64 apply
    dom_key = DOMINANT if (hinfo["outer_pair"] and DOMINANT in kernels) else DOMINANT_FP64
    dom, domh, d64 = kernels[dom_key], kernels[DOMINANT_HBM], kernels[DOMINANT_FP64]

    # end to end through the host-buffer entry point (pinned host memory)
    bh = torch.from_numpy(P.b.reshape(-1).copy()).pin_memory().numpy()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    H.solve_host(bh, xh, tol=TOL, maxit=1000, precision=xdg.XDG_PREC_F32)
    if dist:
        dist.barrier()
    t = time.perf_counter()
    for _ in range(args.steps):
        H.solve_host(bh, xh, tol=TOL, maxit=1000, precision=xdg.XDG_PREC_F32)
    e2e_s = time.perf_counter() - t
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e = job_throughput(world, n, args.steps, e2e_s)

    section_s = {}  # wall seconds of every further section (outside the timed region)

    def timed(name, fn, *a):
        t0 = time.perf_counter()
        r = fn(*a)
        section_s[name] = round(time.perf_counter() - t0, 1)
        return r

    schwarz = None
    if not args.no_schwarz:
        schwarz = timed("schwarz", schwarz_section, xdg, torch, dev, stream, P, xref, args.steps, warmup)

    solvers = None
    if not args.no_solvers:
        solvers = timed("other_solvers", solvers_section, xdg, torch, dev, stream, P, xref)

    learned_out = None
    if not args.no_learned:
        learned_out = timed("learned", learned_section, xdg, torch, dev, stream, 4, budget)

    c3_out = None
    twin = None
    if c3_thread is not None:
        t0 = time.perf_counter()
        c3_thread.join()
        section_s["c3_generation_wait"] = round(time.perf_counter() - t0, 1)
        H.destroy()
        c3_out = timed("c3", c3_section, xdg, torch, dev, stream, c3["P"], c3["R"], c3["gen_s"],
                       min(args.steps, C3_STEPS), args.c3_oracle, not args.no_schwarz)
        c3.pop("P")
        if "twin" in c3:
            twin = timed("paper_twin", twin_section, xdg, torch, dev, stream, c3.pop("twin"))
        c3.clear()

    batched = None
    if not args.no_batch:
        H.destroy()  # free the single problem's hierarchy first
        batched = timed("batched", batched_section, xdg, torch, dev, stream, args.steps, warmup)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        it64 = int(statistics.median(iters64))
        s = oracle_sample(P, it64)
        one = s["single_thread"]
        cpu = {"value": n / s["est_solve_s"] / 1e6, "unit": "MDOF/s", "cores": s["cores"], "kind": "oracle",
               "sample": "%d FP64 PCG iterations of the same 64^3 problem (%.3f s each), extrapolated to the "
                         "%d iterations of the FP64 solve" % (s["sample_iterations"], s["per_iteration_s"], it64),
               "single_thread": {"value": n / one["est_solve_s"] / 1e6, "unit": "MDOF/s", "cores": 1,
                                 "sample": "%d PCG iterations on one thread (%.3f s each), extrapolated the same way"
                                           % (one["sample_iterations"], one["per_iteration_s"])}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer (apply: f32 pairs) / f32 cycle" if hinfo["outer_pair"] else "f64 outer / f32 cycle",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "dof": n, "blocks": nb, "nnz_blocks": nnzb, "Np": Np,
                       "levels": hinfo["nb"], "cycle": "W(1,1) on the 2 finest levels, V below; block Jacobi",
                       "outer": "flexible CG, FP64 residual/update/inner products; apply %s" % (
                           "from FP32 pairs (FP64-accurate, double-float)" if hinfo["outer_pair"] else "in FP64"),
                       "tol": TOL, "iterations": iters,
                       "parallelism": "replicas" if world > 1 else "single",
                       "split_rows_levels": hinfo["split"],
                       "outer_apply_pair": hinfo["outer_pair"],
                       "symmetric_level1": {"cycle": hinfo["symmetric_cycle"], "pair": hinfo["symmetric_pair"]},
                       "fused_small_levels_from": hinfo["fused_level"],
                       "l2": "inputs larger than L2 (operator 1.49 GB FP64 + 0.74 GB FP32)"},
            "paths": {
                "mixed_f32": {"solve_ms": t_ms / args.steps, "iterations": iters, "mdofs": value / world,
                              "rel_l2_vs_oracle": err32},
                "plain_f64": {"solve_ms": t64_ms / args.steps, "iterations": iters64,
                              "mdofs": n * args.steps / (t64_ms / 1e3) / 1e6, "rel_l2_vs_oracle": err64},
                "mixed_bf16_transfers": {"solve_ms": tbf_ms / args.steps, "iterations": itersbf,
                                         "mdofs": n * args.steps / (tbf_ms / 1e3) / 1e6, "rel_l2_vs_oracle": errbf},
                "speedup_mixed_vs_f64": t64_ms / t_ms,
            },
            "parity": {"rel_l2_vs_oracle": {"mixed_f32": err32, "plain_f64": err64, "mixed_bf16_transfers": errbf},
                       "bound": PARITY_BOUND,
                       "oracle": "FP64 PCG on the host cores to relative residual %.0e (%d iterations, %.1f s), "
                                 "outside the timed regions; each path's last timed solution" % (
                                     rr_ref if rr_ref > 0 else 1e-13, it_ref, oracle_s)},
            "vcycle_mdofs": {"f64": n / cyc_ms[0] / 1e3, "f32": n / cyc_ms[1] / 1e3, "bf16": n / cyc_ms[2] / 1e3},
            "vcycle_ms": cyc_ms,
            "setup_s": setup_s, "setup_ms_phases": hinfo["setup_ms"],
            "roofline": (
                {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["achieved_gbs"], "peak": hbm,
                 "unit": "GB/s", "frac": dom["achieved_gbs"] / hbm, "peak_kind": hbm_kind, "bytes": dom["bytes"],
                 "ms": dom["ms"], "traffic": profiled_traffic(dom["name"], dom["bytes"])}
                if dom_key != DOMINANT_FP64 else
                {"bound": "alu", "kernel": dom["kernel"], "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
                 "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS, "flops": flops_apply, "bytes": dom["bytes"],
                 "ms": dom["ms"], "traffic": profiled_traffic(dom["name"], dom["bytes"]),
                 "peak_kind": "FP64 unit counts x clock (152 SMs x 2.07 GHz x 4 flop)"}),
            "roofline_fp64": {"bound": "alu", "kernel": d64["kernel"], "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS,
                              "peak_kind": "FP64 unit counts x clock (152 SMs x 2.07 GHz x 4 flop); the library's "
                                           "FMA probe reaches %.3f TFLOP/s of it" % fp64_peak,
                              "flops": flops_apply, "bytes": d64["bytes"], "ms": d64["ms"],
                              "traffic": profiled_traffic(d64["name"], d64["bytes"])},
            "roofline_hbm": {"bound": "hbm", "kernel": domh["kernel"], "achieved": domh["achieved_gbs"], "peak": hbm,
                             "unit": "GB/s", "frac": domh["achieved_gbs"] / hbm, "peak_kind": hbm_kind,
                             "bytes": domh["bytes"], "ms": domh["ms"],
                             "traffic": profiled_traffic(domh["name"], domh["bytes"])},
            "kernels_level1": kernels,
            "fp64_fma_probe_tflops": fp64_peak,
            "batched": batched,
            "learned": learned_out,
            "schwarz": schwarz,
            "c3_mixed_precision": c3_out,
            "paper_twin": twin,
            "section_wall_s": section_s,
            "other_solvers": solvers,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "MDOF/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    errs = [err32, err64, errbf]
    if schwarz:
        errs += [schwarz["mixed_f32"]["rel_l2_vs_oracle"], schwarz["plain_f64"]["rel_l2_vs_oracle"]]
    if learned_out:
        errs += list(learned_out["rel_l2_vs_oracle"].values())
    if batched:
        errs += list(batched["parity"]["max_rel_l2_vs_oracle"].values())
    if c3_out:
        errs += [v[k] for v in c3_out["paths"].values() for k in ("rel_l2_vs_oracle", "rel_l2_vs_fp64_gpu") if k in v]
    # other solvers: every solve that reports convergence must meet the bound
    if solvers:
        errs += [v["rel_l2_vs_oracle"] for v in solvers.values() if isinstance(v, dict) and v["converged"]]
    if twin:
        errs += [v[t]["rel_l2_vs_fp64_cg"] for v in twin["cases"]
                 for t in ("cg_f32_wcycle", "cg_f64_wcycle", "orthomg_schwarz", "gmres_pmg_klo1", "gmres_pmg_klo3")
                 if t in v and v[t]["converged"]]
    worst = max(errs)
    if worst > PARITY_BOUND:
        print("bench: a timed solution is %.3e from the oracle's (bound %.0e)" % (worst, PARITY_BOUND),
              file=sys.stderr, flush=True)
        sys.exit(1)


if __name__ == "__main__":
    main()
