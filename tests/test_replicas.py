"""Multi-process path of bench.py on CPU (gloo, world size 2): replicas with no data-path
collective; the job time is the slowest rank's and the throughput counts every rank's work;
the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slow = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    dist.barrier()
    q.put((rank, slow))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 15.0, 1: 15.0}


def test_job_throughput_counts_every_replica():
    import bench
    one = bench.job_throughput(1, 2_662_320, 5, 0.4)
    assert abs(bench.job_throughput(2, 2_662_320, 5, 0.4) - 2 * one) < 1e-9
    assert abs(one - 2_662_320 * 5 / 0.4 / 1e6) < 1e-9


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "make_problem", lambda: called.append(1))
    bench.reference_arm(argparse.Namespace(steps=1, warmup=1))
    assert not called and capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract():
    """bench.py --impl reference prints one JSON line with the benchmark's keys, the oracle's
    cpu_baseline (its value the line's) and an e2e entry without host-device copies."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.pop("RANK", None)
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--size", "12",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"].startswith("xdg-poisson-3d-12^3")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # ms_per_step is the measured step (the sample); value extrapolates it to the full solve
    assert d["extrapolated_solve_ms"] >= d["ms_per_step"] > 0
    assert abs(d["value"] - d["config"]["dof"] / d["extrapolated_solve_ms"] / 1e3) <= 1e-9 * d["value"]
