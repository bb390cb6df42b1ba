"""Host logic of bench.py on CPU: the throttle-reason summary of the sampled clocks and the
guard that reports the fused kernel's measured DRAM traffic only for the sources measured."""
import importlib.util
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


def test_clock_summary_median_and_reasons(bench):
    c = bench.ClockSampler(0)
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line",
               "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["0, 1500, 2070, 800, 0x20, Not Active, Active, Not Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_traffic_reported_only_for_the_measured_sources_and_shape(bench, monkeypatch):
    t = bench.FUSED_TRAFFIC
    cfg = types.SimpleNamespace(tile=t["tile"], ppt=t["ppt"], batch=t["batch"])
    got = bench.fused_traffic(cfg, bench.N_GAUSS, bench.N_VIEWS)
    assert got in (t["bytes"], None)          # None once a hashed source has changed
    assert bench.fused_traffic(types.SimpleNamespace(tile=16, ppt=1, batch=1), bench.N_GAUSS, bench.N_VIEWS) is None
    # batch 2 runs the CTA kernel, not the one measured
    assert bench.fused_traffic(types.SimpleNamespace(tile=32, ppt=2, batch=2), bench.N_GAUSS, bench.N_VIEWS) is None
    assert bench.fused_traffic(cfg, 300_000, 8) is None
    monkeypatch.setitem(bench.FUSED_TRAFFIC, "sha256", "0" * 64)
    assert bench.fused_traffic(cfg, bench.N_GAUSS, bench.N_VIEWS) is None
