"""Host-side logic of bench.py (no GPU): the DRAM traffic it reports is read from a committed
ncu summary only while the CUDA sources hash to the digest recorded there, scaled by the
algorithmic bytes; the performance-study tables are consistent with each other and with the
paper's DOF table."""
import os

import pytest

import bench


def _fake_root(tmp_path, src="kernel A"):
    csrc = tmp_path / "paper_2003_02431_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text(src)
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_traffic_read_only_for_matching_sources_and_scaled(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    digest = bench.csrc_digest()
    (root / "profiles" / "k.md").write_text(
        "text\ntraffic_per_launch kernel=k_x<10> size=48 bytes=400 alg_bytes=200 csrc_sha256=%s\n" % digest)
    assert bench.profiled_traffic("k_x<10>", 200) == 400
    assert bench.profiled_traffic("k_x<10>", 1000) == 2000      # scaled by the algorithmic bytes
    assert bench.profiled_traffic("k_y<10>", 200) is None       # another kernel
    (root / "paper_2003_02431_gb300" / "csrc" / "a.cu").write_text("kernel A, changed")
    assert bench.csrc_digest() != digest
    assert bench.profiled_traffic("k_x<10>", 200) is None       # stale counters are not reported


def test_digest_depends_on_names_and_contents(tmp_path, monkeypatch):
    root = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    d0 = bench.csrc_digest()
    os.rename(root / "paper_2003_02431_gb300" / "csrc" / "a.cu", root / "paper_2003_02431_gb300" / "csrc" / "b.cu")
    assert bench.csrc_digest() != d0


def test_performance_study_tables_are_consistent():
    table = bench.paper_dof_table()
    for k, N in bench.TWIN_CASES:
        assert (k, N) in table, (k, N)            # every case is compared with the paper's count
    for k, N in bench.TWIN_CASES:
        for klo in bench.PMG_KLO[k]:
            assert klo < k and (k, klo) in bench.TWIN_PMG_MAXIT
            assert bench.N_LO_3D[klo] == (klo + 1) * (klo + 2) * (klo + 3) // 6   # dim of P_klo in 3D
    for k, N in bench.TWIN_PMG_N.items():
        assert (k, N) in bench.TWIN_CASES


@pytest.mark.parametrize("world,units,steps,seconds,expect", [(1, 2e6, 10, 1.0, 20.0), (4, 1e6, 2, 0.5, 16.0)])
def test_job_throughput(world, units, steps, seconds, expect):
    assert bench.job_throughput(world, units, steps, seconds) == pytest.approx(expect)
