"""CPU tests of bench.py's host-side helpers: the clock sampler's bookkeeping
(driven by a stand-in for nvidia-smi that prints CSV rows every 20 ms)."""
import sys
import time

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402

FAKE = ("import sys, time\n"
        "i = 0\n"
        "while True:\n"
        "    r = 'Active' if i == {throttle} else 'Not Active'\n"
        "    print('0, %d, 2070, Not Active, %s, Not Active, Not Active' % (1900 + i, r), flush=True)\n"
        "    i += 1\n"
        "    time.sleep(0.02)\n")


def _sampler(throttle=-1):
    return bench.ClockSampler(0, argv=[sys.executable, "-c", FAKE.format(throttle=throttle)])


def test_clock_sampler_keeps_samples_of_the_timed_region():
    c = _sampler()
    c.start()
    assert c._lines, "start returns only once sampling is live"
    time.sleep(0.2)
    out = c.stop()
    # ~10 samples inside a 200 ms region, plus the one before it
    assert 6 <= out["samples"] <= 14
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []
    assert out["timed_region_s"] == pytest.approx(0.2, abs=0.05)
    assert 1900 <= out["sm_mhz"] <= 1900 + 30


def test_clock_sampler_short_region_brackets_it():
    c = _sampler()
    c.start()
    out = c.stop()                   # a region far shorter than the period
    assert 1 <= out["samples"] <= 2
    assert out["sm_mhz"] is not None


def test_clock_sampler_reports_throttle_reasons():
    c = _sampler(throttle=0)         # the first sample shows hw_thermal_slowdown
    c.start()
    time.sleep(0.1)
    out = c.stop()
    assert out["reasons"] == ["hw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler(0, argv=["/nonexistent/nvidia-smi"])
    c.start()
    assert c.stop()["reasons"] == ["unsampled"]


def test_clock_sampler_falls_back_to_a_longer_period():
    # a stand-in that exits at once when asked for a 20 ms period
    prog = ("import sys, time\n"
            "if sys.argv[1] == '20': sys.exit(2)\n" + FAKE.format(throttle=-1).split("\n", 1)[1])
    c = bench.ClockSampler(0, argv=[sys.executable, "-c", prog, "20"])
    c.start()
    time.sleep(0.25)
    out = c.stop()
    assert out["period_ms"] == 100 and out["samples"] >= 1


def test_algorithmic_bytes_per_precision():
    info1 = {"nf1": 2000, "nf2": 2000}
    info3 = {"nf1": 1500, "nf2": 1400, "nfft1": 3000, "nfft2": 2800}
    a32 = bench.algorithmic_bytes(info1, info3, 524288)
    a64 = bench.algorithmic_bytes(info1, info3, 524288, "fp64")
    assert a32["t3.spread"] == 524288 * 24 + 1500 * 1400 * 8
    assert a64["t3.spread"] == 524288 * 40 + 1500 * 1400 * 16
    assert a32["t3.interp_epilogue"] == bench.M3 * 24
    assert a64["t3.interp_epilogue"] == bench.M3 * 32
    assert set(a32) == set(a64)
    # a pruned type-1 plan moves only its live rows (here 40 tile rows of 32)
    a = bench.algorithmic_bytes(dict(info1, live_tile_rows=40, tile_y=32), info3, 524288)
    assert a["t1.spread"] == 524288 * 24 + 2000 * 1280 * 8
    assert a["t1.fft_cols_epilogue"] == (1000 * 1280 + 1000 * 1000) * 8
    assert bench.live_rows({"live_tile_rows": 0}, 777) == 777


def test_precision_option_is_star_only():
    import subprocess
    r = subprocess.run([sys.executable, bench.__file__, "--workload", "starshade_sweep",
                        "--precision", "fp64"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "star5_F100" in r.stderr


def test_rel_error_reports_l2_max_and_tolerance():
    import numpy as np
    ref = np.array([1.0 + 1.0j, -2.0, 0.5j, 3.0])
    u = ref + np.array([1e-7, 0.0, -2e-7j, 0.0])
    e = bench.rel_error(u, ref, 1e-6)
    assert e["rel_l2"] == pytest.approx(np.sqrt(5e-14) / np.linalg.norm(ref))
    assert e["max_abs"] == pytest.approx(2e-7)
    assert e["oracle_targets"] == 4 and e["within_tol"]
    assert not bench.rel_error(ref * (1 + 1e-5), ref, 1e-6)["within_tol"]
    # an occulter field is graded on u^ap = 1 - u^oc: a small u^oc keeps its
    # absolute error but not its relative one
    oc = np.array([1e-3, -2e-3j, 1.5e-3])
    e = bench.rel_error(oc + 1e-7, oc, 1e-6, occulter=True)
    assert e["within_tol"] and e["field"].startswith("u^ap")
    assert not bench.rel_error(oc + 1e-7, oc, 1e-6)["within_tol"]


def test_traffic_is_dropped_when_the_kernel_sources_change(monkeypatch):
    sha = bench.sources_sha("spread")
    monkeypatch.setitem(bench.DRAM_TRAFFIC, ("w", "t3.spread"),
                        bench._cap(123, 0.5, 0.4, 0.7, sha, "capture"))
    b, why, sm = bench.measured_traffic("w", "t3.spread")
    assert (b, why) == (123, "capture") and sm["issue_slots_busy"] == 0.5
    monkeypatch.setitem(bench.DRAM_TRAFFIC, ("w", "t3.spread"),
                        bench._cap(123, 0.5, 0.4, 0.7, "0" * 16, "capture"))
    b, why, sm = bench.measured_traffic("w", "t3.spread")
    assert b is None and sm is None and "changed" in why
    assert bench.measured_traffic("w", "t1.fft_rows")[0] is None


def test_roofline_picks_the_slowest_stage_with_bytes():
    r = bench.roofline("w", {"a.spread": 4e9, "a.fft_rows": 1e9},
                       {"a.spread": 2.0, "a.fft_rows": 1.0, "a.scan": 5.0}, "note")
    assert r["kernel"] == "a.spread"
    assert r["achieved"] == pytest.approx(4e9 / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_capture_table_entries_are_well_formed():
    """Every traffic entry carries its bytes, SM-side utilisations (fractions
    of their own peaks), a source hash and a note; entries whose kernel
    sources changed report null (measured_traffic)."""
    for (wl, stage), e in bench.DRAM_TRAFFIC.items():
        assert bench.stage_kind(stage) in bench.KERNEL_SOURCES
        assert e["bytes"] > 0 and e["note"] and len(e["sources_sha"]) == 16
        assert all(0 < v <= 1 for v in e["sm_side"].values())
