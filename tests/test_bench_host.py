"""Host logic of bench.py that needs no GPU: the clock summary taken during the timed region,
the validity check of the committed ncu traffic record, the iteration count the oracle legs take
from the committed bench record, and the oracle leg itself on a small problem."""
import json
import os

import numpy as np
import pytest

import bench


def test_clock_summary_median_and_reasons():
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2040, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
    ]
    s = bench.summarize_clock_rows(rows)
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_flags_thermal_and_hw_slowdown():
    rows = ["0, 1500, 2070, 1000, 0x48, Active, Not Active, Active, Not Active\n"] * 2
    s = bench.summarize_clock_rows(rows)
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_without_samples_is_none():
    assert bench.summarize_clock_rows([]) is None
    assert bench.summarize_clock_rows(["[N/A]\n"]) is None


def test_traffic_record_is_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    key = "cgloop_fp32|logistic_20000x8000"
    assert key in rec and rec[key]["dram_bytes_per_iteration"] > 0
    # a record for other sources is not used
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / "ncu_traffic.json").write_text(json.dumps(
        {key: {"source_hash": "0" * 16, "dram_bytes_per_iteration": 1.0}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "cgloop_source_hash", lambda: "f" * 16)
    assert bench.traffic_record("cgloop_fp32", "logistic_20000x8000") is None
    monkeypatch.setattr(bench, "cgloop_source_hash", lambda: "0" * 16)
    assert bench.traffic_record("cgloop_fp32", "logistic_20000x8000") == 1.0
    assert bench.traffic_record("cgloop_fp32", "other") is None


def test_recorded_iteration_count_comes_from_the_committed_bench_record(tmp_path, monkeypatch):
    its, rec = bench.recorded_iterations("logistic_20000x8000")
    assert rec == os.path.join("profiles", "bench_logistic_20000x8000.json")
    committed = json.load(open(os.path.join(bench.ROOT, rec)))["solve"]["iters"]
    assert its == int(np.median(committed)) and its > 0
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "bench_w.json").write_text(json.dumps({"solve": {"iters": [10, 30, 20]}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_iterations("w")[0] == 20
    assert bench.recorded_iterations("missing")[0] is None


def test_blas_threads_follow_the_environment(monkeypatch):
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.delenv(k, raising=False)
    assert bench.blas_threads() == os.cpu_count()
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    assert bench.blas_threads() == 3


def test_oracle_leg_certifies_z_and_times_an_iteration():
    """The cpu_baseline leg on a small Lasso: the oracle's float64 rel-KKT of a given z, and a
    value equal to the timed seconds per exact iteration times the count passed in."""
    import problems
    from oracle import admm, checks
    P = problems.lasso_iid(60, 120, nnz=6, seed=3)
    lam = 0.1 * checks.lambda_max(P.A, P.b, "squared")
    ref = admm.solve(P.A, P.b, "squared", lam, tol=1e-10)
    leg = bench.oracle_leg(P, lam, 1.0, ref["z"], iters=50, sample_iters=2)
    assert leg["rel_kkt_oracle"] <= 1e-10
    assert leg["value"] == leg["per_iter_s"] * 50 and leg["per_iter_s"] > 0
    assert leg["kind"] == "oracle" and leg["cores"] >= 1 and "x 50 iterations" in leg["sample"]
    bad = bench.oracle_leg(P, lam, 1.0, np.zeros(P.n), iters=1, sample_iters=1)
    assert bad["rel_kkt_oracle"] > 1e-3     # z = 0 is not the solution below lambda_max


def test_record_traffic_parses_ncu_csv_and_keys_by_source_hash(tmp_path, monkeypatch):
    """The traffic record is (dram read + write bytes of the cgloop launch) / iterations, keyed by
    the current hash of the kernel's sources; other kernels' rows are ignored."""
    csvf = tmp_path / "cap.csv"
    csvf.write_text(
        '==PROF== Connected\n'
        '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
        '"0","1","python","h","void genios::cgloop_kernel<1, 4>(CgLoopArgs, int, int)","1","7","(544, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Gbyte","12.83"\n'
        '"0","1","python","h","void genios::cgloop_kernel<1, 4>(CgLoopArgs, int, int)","1","7","(544, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Mbyte","50.80"\n'
        '"1","1","python","h","void genios::rowpass_kernel<1, 4, 1>(RowpassArgs, int, int)","1","7","(544, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Gbyte","0.64"\n')
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "cgloop_source_hash", lambda: "a" * 16)
    rec = bench.record_traffic(str(csvf), 20)
    assert rec["source_hash"] == "a" * 16
    assert rec["dram_bytes_per_iteration"] == pytest.approx((12.83e9 + 50.8e6) / 20)
    assert bench.traffic_record("cgloop_fp32", "logistic_20000x8000") == pytest.approx(rec["dram_bytes_per_iteration"])


def test_record_traffic_reads_the_raw_page_export(tmp_path, monkeypatch):
    """The same record from ncu's raw-page CSV export (one column per metric, units in row 2)."""
    csvf = tmp_path / "raw.csv"
    csvf.write_text(
        '"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum","gpu__time_duration.sum"\n'
        '"","","Mbyte","Kbyte","msecond"\n'
        '"0","void genios::cgloop_kernel<1, 4>(CgLoopArgs, int, int)","12,833.10","50,800.00","2.11"\n')
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "cgloop_source_hash", lambda: "b" * 16)
    rec = bench.record_traffic(str(csvf), 20)
    assert rec["dram_bytes_per_iteration"] == pytest.approx((12833.1e6 + 50.8e6) / 20)
