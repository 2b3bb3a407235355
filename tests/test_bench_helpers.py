"""Host logic of bench.py (no GPU): the clock summary that decides whether a
timed run is kept, the guard that ties the recorded walk traffic to the walk
source it was measured on, the peak denominators and the shared workload
description of both arms."""
import hashlib
import os

import pytest

import bench


def _sample(t, sm, mx, hw=False, therm=False, swtherm=False, cap=False):
    flag = lambda x: "Active" if x else "Not Active"
    return (t, [str(sm), str(mx), "900.0", "0x0", flag(hw), flag(therm), flag(swtherm), flag(cap)])


def test_clock_summary_uses_the_timed_window():
    c = bench.ClockSampler(0)
    c.samples = [_sample(0.0, 1200, 2070, therm=True),  # warm-up, outside the window
                 _sample(1.00, 2070, 2070), _sample(1.02, 2055, 2070, cap=True), _sample(1.04, 2070, 2070),
                 _sample(5.0, 900, 2070, hw=True)]  # after the window
    c.window(0.99, 1.05)
    s = c.summary()
    assert s["sampled"] == "timed region" and s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]  # the thermal and hw events outside the window do not count


def test_clock_summary_reports_throttling_inside_the_window():
    c = bench.ClockSampler(0)
    c.samples = [_sample(2.0, 1500, 2070, hw=True, swtherm=True), _sample(2.01, 1480, 2070, therm=True)]
    c.window(1.99, 2.02)
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1490.0


def test_clock_summary_without_samples_in_the_window():
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["unsampled"]
    c.samples = [_sample(0.0, 2000, 2070), _sample(10.0, 1000, 2070)]
    c.window(1.0, 1.001)  # a region shorter than the sampling period: the nearest sample
    s = c.summary()
    assert s["sampled"] == "nearest to the timed region" and s["sm_mhz"] == 2000.0


def test_walk_traffic_only_for_the_captured_source(monkeypatch):
    path = os.path.join(bench.ROOT, "paper_1909_04667_gb300", "csrc", "walk.cu")
    digest = hashlib.sha256(open(path, "rb").read()).hexdigest()
    same = dict(bench.WALK_TRAFFIC, walk_cu_sha256=digest)
    monkeypatch.setattr(bench, "WALK_TRAFFIC", same)
    assert bench.walk_capture() is same
    monkeypatch.setattr(bench, "WALK_TRAFFIC", dict(same, walk_cu_sha256="0" * 64))
    assert bench.walk_capture() is None
    # the recorded figures are per launch: DRAM bytes of one walk and the executed FP32 rate
    assert 1e7 < same["bytes"] < 1e9 and 0 < same["fma_pipe_active"] <= 1 and 0 < same["alu_pipe_inst"] <= 1


def test_peaks_measured_or_fallback():
    pk, kind = bench.peaks()
    assert kind in ("measured", "fallback")
    assert pk["hbm_gbs"] > 1000 and pk["sm_max_mhz"] > 1000


@pytest.mark.parametrize("world", [1, 4])
def test_headline_config_names_the_workload(world):
    c = bench.headline_config(world)
    assert c["workload"] == "hernquist_n2^20_relative_alpha0.0025"
    assert c["n_particles"] == c["n_active"] == c["global_batch"] == 1 << 20
    assert c["parallelism"] == ("replicas" if world > 1 else "single")
    assert "model" not in c and "l2" in c
