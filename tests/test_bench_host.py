"""Host logic of bench.py that needs no GPU: the clock summary taken during the timed region,
the validity check of the committed ncu traffic record, and the reduced problem used for the
oracle's iteration count."""
import json
import os

import numpy as np

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


def test_reduced_problem_keeps_the_generator_and_scales_by_eight():
    P = bench.make_problem("lasso_1000x10000")
    R = bench.reduced_problem(P, 77)
    assert (R.m, R.n, R.loss) == (P.m // 8, P.n // 8, P.loss)
    assert np.all(np.isfinite(R.A)) and R.A.shape == (R.m, R.n)
