"""Host-side bookkeeping of bench.py (no GPU): the workload label follows the
sizes actually run, committed ncu traffic figures are reported only for the
workload they were taken on, and the ALU peak's clock is read from the
measured peaks (or the GB300 maximum)."""
import importlib.util
import json
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_workload_label_follows_the_sizes(bench):
    a = types.SimpleNamespace(n=200_000, dim=960, nq=2_000, k=10, M=20)
    name = bench.workload_name(a)
    assert "N=200,000" in name and "D=960" in name and "2,000 held-out queries" in name and "M=20" in name


def test_traffic_only_for_its_workload(bench):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    w = dict(d["workload"])
    for stage, v in d["bytes_per_launch"].items():
        assert bench._ncu_traffic(stage, w) == v
    assert bench._ncu_traffic("no such stage", w) is None
    other = dict(w, N=w["N"] // 5)
    assert all(bench._ncu_traffic(stage, other) is None for stage in d["bytes_per_launch"])
    # every committed figure is a plausible per-launch byte count for that workload
    for v in d["bytes_per_launch"].values():
        assert 1e8 < v < 1e12


def test_max_sm_clock_for_the_alu_peak(bench):
    # the ALU peak is SMs x 128 FP32 lanes x 2 flops x this clock
    mhz = bench.max_sm_mhz()
    assert 1000 <= mhz <= 3000
