#!/usr/bin/env python3
"""Benchmark of the multigrid-preconditioned XDG solve on GB300 (libxdg through its C ABI).

Workload (synthetic, generated in-process): 3D XDG Poisson problem on the unit cube, 64^3
Cartesian cells, spherical interface (centre (0.5,0.5,0.5), radius 0.31), diffusivity 1 inside /
1000 outside, SIP, DG degree k=2 (Np=10), agglomeration threshold 0.1, manufactured smooth
solution: 266,232 blocks, 2,662,320 DOF, 1,849,256 non-zero 10x10 blocks.

A step is one complete solve from x = 0: conjugate gradients preconditioned by the symmetric
W-cycle (block-Jacobi smoothing, fused residual-restriction, prolongation, dense coarsest
solve), stopped at ||b - M x|| <= 1e-10 ||b|| (the parity tests show the solution then lies
within 1e-8 relative L2 of the FP64 oracle's solution). value = DOF solved per second.

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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "XDG solve time to 1e-8 rel. L2 & V-cycle MDOF/s vs plain FP64 path, 1 GB300"
WORKLOAD = "xdg-poisson-3d-64^3-k2-sphere-R0.31-mu1:1000"
TOL = 1e-10


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def make_problem():
    import xdg_problem as xp
    return xp.Problem(xp.config_3d_64(max_coarse_dof=1000))


def oracle_sample(P, iters_needed, budget_s=12.0):
    """Time the oracle's PCG iterations on this problem (bounded sample) and extrapolate."""
    import oracle
    t = time.perf_counter()
    O = oracle.Hierarchy(P, gamma=2)
    setup = time.perf_counter() - t
    m, spent, per = 4, 0.0, None
    while True:
        t = time.perf_counter()
        O.pcg(P.b, tol=0.0, maxit=m)
        dt = time.perf_counter() - t
        per = dt / m
        spent += dt
        if dt >= budget_s / 3 or spent >= budget_s:
            break
        m *= 2
    est = per * iters_needed
    return {"per_iteration_s": per, "sample_iterations": m, "setup_s": setup, "est_solve_s": est,
            "cores": os.cpu_count()}


def reference_arm(args):
    """The oracle (plain FP64 CPU) on the same workload: each step a bounded sample of PCG
    iterations; the metric extrapolates with the iteration count the oracle needs."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    P = make_problem()
    O = oracle.Hierarchy(P, gamma=2)
    _, iters, _, _ = O.pcg(P.b, tol=TOL, maxit=1000)  # warm-up: a full solve gives the count
    per = []
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        O.pcg(P.b, tol=0.0, maxit=5)
        if s >= args.warmup:
            per.append((time.perf_counter() - t) / 5)
    t_iter = statistics.mean(per)
    t_solve = t_iter * iters
    value = P.dof / t_solve / 1e6
    line = {"metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "dof": P.dof, "tol": TOL, "iterations": iters,
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "5 PCG+W-cycle iterations per step, extrapolated to the %d "
                                       "iterations of the full solve" % iters},
            "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xdg", choices=["xdg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
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
    stream = torch.cuda.Stream(device=dev)   # the handle's stream; events are recorded on it

    P = make_problem()
    n = P.dof
    t = time.perf_counter()
    H = xdg.Hierarchy.from_problem(P, gamma=2, stream=stream)
    setup_s = time.perf_counter() - t
    hinfo = H.info()
    b = torch.from_numpy(P.b.reshape(-1).copy()).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)

    def solve():
        x.zero_()
        return H.solve(b, x, tol=TOL, maxit=1000)

    for _ in range(max(args.warmup, 3)):
        info = solve()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches, iters = 0, []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            info = solve()
            launches += info["launches"]
            iters.append(info["iterations"])
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_ms = ev0.elapsed_time(ev1)
    if dist:
        tt = torch.tensor([t_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    value = world * n * args.steps / (t_ms / 1e3) / 1e6

    # one cycle alone (graph replay), CUDA events on the same stream
    z = torch.empty_like(x)
    for _ in range(3):
        H.vcycle(b, z)
    nv = 20
    ev0.record(stream)
    for _ in range(nv):
        H.vcycle(b, z)
    ev1.record(stream)
    torch.cuda.synchronize()
    cycle_ms = ev0.elapsed_time(ev1) / nv

    # dominant kernels on level 1, CUDA events on the launching stream
    Np, nb, nnzb = P.Np, P.nb[0], int(P.row_ptr[-1])
    bytes_apply = nnzb * (Np * Np * 8 + 4) + (nb + 1) * 8 + 2 * n * 8
    bytes_smooth = bytes_apply + nb * (Np * (Np + 1) // 2) * 8 + 2 * n * 8
    bytes_restrict = bytes_apply - n * 8 + nb * (Np * Np * 8 + 8) + n * 8 + P.nb[1] * Np * 8 + (P.nb[1] + 1) * 8
    y = torch.empty_like(x)

    def time_kernel(fn, reps=20):
        for _ in range(3):
            fn()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    rc = torch.empty(P.nb[1] * Np, dtype=torch.float64, device=dev)
    k_ms = {"apply": time_kernel(lambda: H.apply(1, b, y)),
            "smooth": time_kernel(lambda: H.smooth(1, b, z, y)),
            "restrict": time_kernel(lambda: H.restrict(1, b, z, rc))}
    k_bytes = {"apply": bytes_apply, "smooth": bytes_smooth, "restrict": bytes_restrict}
    peak, peak_kind = peaks()
    dom = "restrict"
    achieved = k_bytes[dom] / (k_ms[dom] / 1e3) / 1e9

    # end to end through the host-buffer entry point (pinned host memory)
    bh = torch.from_numpy(P.b.reshape(-1).copy()).pin_memory().numpy()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    H.solve_host(bh, xh, tol=TOL, maxit=1000)
    if dist:
        dist.barrier()
    t = time.perf_counter()
    for _ in range(args.steps):
        H.solve_host(bh, xh, tol=TOL, maxit=1000)
    e2e_s = time.perf_counter() - t
    if dist:
        tt = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e = world * n * args.steps / e2e_s / 1e6

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_sample(P, int(statistics.median(iters)))
        cpu = {"value": n / s["est_solve_s"] / 1e6, "unit": "MDOF/s", "cores": s["cores"], "kind": "oracle",
               "sample": "%d PCG+W-cycle iterations of the same 64^3 problem (%.2f s/iteration), "
                         "extrapolated to the %d iterations of the GPU solve"
                         % (s["sample_iterations"], s["per_iteration_s"], int(statistics.median(iters)))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dof": n, "blocks": nb, "nnz_blocks": nnzb, "Np": Np,
                       "levels": hinfo["nb"], "cycle": "W(1,1) block-Jacobi", "tol": TOL,
                       "iterations": iters, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (operator 1.49 GB)"},
            "vcycle_mdofs": n / (cycle_ms / 1e3) / 1e6, "vcycle_ms": cycle_ms,
            "setup_s": setup_s, "setup_ms_phases": hinfo["setup_ms"],
            "kernels_ms": k_ms,
            "kernels_gbs": {k: k_bytes[k] / (k_ms[k] / 1e3) / 1e9 for k in k_ms},
            "roofline": {"bound": "hbm", "kernel": "k_restrict (fused residual + restriction, level 1)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": None},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "MDOF/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
