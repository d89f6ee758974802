"""Host logic of the relative-KKT check schedule (KktSchedule in csrc/internal.h), compiled with
g++ on the CPU: a check when the residual test of §2.3 first passes, periodic checks at most
kkt_check_every apart, and earlier checks when the decrease between the last two checks predicts
that the tolerance will be reached sooner."""
import math
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_08333_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROG = r'''
#include <cstdio>
#include "internal.h"
int main() {
    using genios::KktSchedule;
    // (a) periodic: every 10 iterations from the last check at k = 1, no residual pass
    {
        KktSchedule s(10, 1);
        for (int k = 2; k <= 35; ++k)
            if (s.due(k, false)) { std::printf("a %d\n", k); s.record(k, 1.0, 1e-4); }
    }
    // (b) the residual test first passing at k = 5 triggers one check; staying true does not
    {
        KktSchedule s(10, 1);
        for (int k = 2; k <= 20; ++k)
            if (s.due(k, k >= 5)) { std::printf("b %d\n", k); s.record(k, 1.0, 1e-4); }
    }
    // (c) prediction: a residual falling by 10x every 10 iterations from 1e-2 at k = 11 reaches
    // 1e-4 at k = 31; the checks tighten toward it
    {
        KktSchedule s(10, 1);
        for (int k = 2; k <= 40; ++k) {
            if (s.due(k, false)) {
                const double v = 1e-2 * std::pow(10.0, -(k - 11) / 10.0);
                std::printf("c %d %.6e\n", k, v);
                s.record(k, v, 1e-4);
                if (v <= 1e-4) break;
            }
        }
    }
    // (d) a residual that grows keeps the periodic interval
    {
        KktSchedule s(10, 1);
        double v = 1e-3;
        for (int k = 2; k <= 45; ++k)
            if (s.due(k, false)) { std::printf("d %d\n", k); s.record(k, v, 1e-4); v *= 2.0; }
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def out():
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        open(src, "w").write(PROG)
        exe = os.path.join(d, "t")
        subprocess.run(["g++", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, src, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()
    res = {}
    for ln in lines:
        tag, *rest = ln.split()
        res.setdefault(tag, []).append(rest)
    return res


def test_periodic_checks(out):
    assert [int(r[0]) for r in out["a"]] == [11, 21, 31]


def test_first_residual_pass_triggers_one_check(out):
    assert [int(r[0]) for r in out["b"]] == [5, 15]


def test_prediction_tightens_toward_the_tolerance(out):
    ks = [int(r[0]) for r in out["c"]]
    vs = [float(r[1]) for r in out["c"]]
    assert ks[0] == 11 and ks[1] == 21           # no rate before two checks
    assert vs[-1] <= 1e-4 * (1 + 1e-9)           # it stops at a value within the tolerance
    assert ks[-1] == 31                          # exactly where the linear rate reaches it
    assert all(b - a <= 10 for a, b in zip(ks, ks[1:]))


def test_growing_residual_keeps_the_period(out):
    assert [int(r[0]) for r in out["d"]] == [11, 21, 31, 41]


def test_rate_formula_matches_closed_form():
    # the prediction of (c) written out: rate per iteration and iterations to reach eps
    v0, v1, k0, k1, eps = 1e-2, 1e-3, 11, 21, 1e-4
    rate = math.log(v1 / v0) / (k1 - k0)
    assert math.ceil(math.log(eps / v1) / rate) == 10
