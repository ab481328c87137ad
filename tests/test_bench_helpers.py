"""Host logic of bench.py that needs no GPU: the clock record kept beside a
timed region (only samples inside the window count; throttle reasons are
collected; a run with no samples says so) and the k-means line's rooflines."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def line(sm, mx, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return "0, %d, %d, 900.0, 0x0, %s" % (sm, mx, ", ".join(flags))


def test_clock_summary_counts_only_the_timed_window(bench):
    cs = bench.ClockSampler(0)
    cs.lines = [(0.5, line(1000, 2070, ["hw_slowdown"])),       # before the window: ignored
                (1.0, line(2070, 2070)), (1.2, line(2040, 2070, ["sw_power_cap"])), (1.4, line(2070, 2070)),
                (3.0, line(500, 2070, ["sw_thermal_slowdown"]))]  # after the window: ignored
    cs.mark(0.9, 2.0)
    s = cs.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_without_samples(bench):
    cs = bench.ClockSampler(0)
    cs.lines = [(0.1, "garbled"), (0.2, line(2070, 2070))]
    cs.mark(1.0, 2.0)
    assert cs.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_kmeans_line_rooflines(bench):
    units = 2_000_000 * 256 * 60
    peaks = {"bf16_tflops": 1889.1, "hbm_gbs": 6761.6, "sm_max_mhz": 2070.0}
    k = bench.kmeans_line((0.8, 1.0, (2_000_000, 12_000, 300)), (3.8, 4.1, (0, 0, 0)), units,
                          2_000_000 * 61 * 4, peaks, "measured")
    assert k["pass_ms"] == 0.8 and k["deferred_per_sample"] == pytest.approx(0.006)
    r = k["roofline"]
    assert r["bound"] == "tensor" and r["achieved"] == pytest.approx(2 * units / 0.8e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1889.1)
    assert k["hbm"]["frac"] == pytest.approx(2_000_000 * 61 * 4 / 0.8e-3 / 1e9 / 6761.6)
    alu = k["cuda_core_form"]["roofline"]
    assert alu["bound"] == "alu" and alu["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
