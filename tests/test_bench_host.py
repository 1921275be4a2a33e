"""Host-side arithmetic of the benchmark's report (no GPU): the roofline
entry of the dominant kernel class, the per-class rates, the traffic figure
that is reported only for the kernel source it was measured on, and the
in-range tap count that the FLOP figures rest on."""
import importlib.util
import os

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _stats(blur_ms, blur_flops, blur_bytes, assign_ms, assign_bytes):
    z = {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0}
    return {"kernels": {"prep": dict(z), "gather": dict(z),
                        "blur_cols": {"launches": 10, "ms": blur_ms, "bytes": blur_bytes, "flops": blur_flops},
                        "assign": {"launches": 10, "ms": assign_ms, "bytes": assign_bytes, "flops": 0.0}}}


def test_alu_bound_dominant_class(bench):
    peaks = {"hbm_gbs": 6784.5}
    # two steps: 30 ms of target passes at 40 TFLOP/s over 6 GB, 10 ms of assignment
    st = [_stats(15.0, 6e11, 3e9, 5.0, 1e10)] * 2
    rl, per = bench.roofline(st, peaks, "measured", {"sm_max_mhz": 2070.0}, "3dgs-1024")
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert rl["kernel"] == "blur_cols" and rl["bound"] == "alu" and rl["unit"] == "TFLOP/s"
    assert rl["achieved"] == pytest.approx(40.0, abs=1e-3)
    assert rl["peak"] == pytest.approx(peak, abs=0.01)
    assert rl["frac"] == pytest.approx(40.0 / peak, abs=1e-4)
    assert rl["launches"] == 20 and rl["avg_launch_us"] == pytest.approx(1500.0)
    assert rl["share"] == pytest.approx(0.75)
    assert per["assign"]["GB/s"] == pytest.approx(2000.0)
    assert per["blur_cols"]["TFLOP/s"] == pytest.approx(40.0)
    assert per["prep"]["GB/s"] is None


def test_hbm_bound_when_bytes_dominate(bench):
    peaks = {"hbm_gbs": 6000.0}
    # the assignment dominates the time and has no flops: bound by HBM
    st = [_stats(1.0, 1e9, 1e8, 9.0, 4.5e10)]
    rl, _ = bench.roofline(st, peaks, "measured", None, "3dgs-1024")
    assert rl["kernel"] == "assign" and rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert rl["achieved"] == pytest.approx(5000.0)
    assert rl["frac"] == pytest.approx(5000.0 / 6000.0, abs=1e-4)
    assert rl["traffic"] is None  # no measured traffic for this class


def test_traffic_only_for_the_measured_source(bench, monkeypatch):
    st = [_stats(15.0, 6e11, 3e9, 5.0, 1e10)]
    key = ("blur_cols", "3dgs-1024")
    rec = bench.NCU_TRAFFIC[key]
    rl, _ = bench.roofline(st, {"hbm_gbs": 6784.5}, "measured", None, "3dgs-1024")
    assert rl["traffic"] == (rec["bytes_per_launch"] if rec["src"] == bench._kernel_hash() else None)
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, {"bytes_per_launch": 123, "src": "not-this-source"})
    rl, _ = bench.roofline(st, {"hbm_gbs": 6784.5}, "measured", None, "3dgs-1024")
    assert rl["traffic"] is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, {"bytes_per_launch": 123, "src": bench._kernel_hash()})
    rl, _ = bench.roofline(st, {"hbm_gbs": 6784.5}, "measured", None, "3dgs-1024")
    assert rl["traffic"] == 123


@pytest.mark.parametrize("length,r", [(1, 0), (7, 3), (16, 15), (100, 7), (1024, 511), (37, 36)])
def test_pass_fmas_counts_in_range_taps(bench, length, r):
    D, other = 5, 3
    brute = sum(1 for p in range(length) for j in range(-r, r + 1) if 0 <= p + j < length)
    assert bench.pass_fmas(length, r, other, D) == brute * other * D
    # the closed form the device counters use: len (2r + 1) - r (r + 1)
    assert brute == length * (2 * r + 1) - r * (r + 1)


def test_clock_sampler_parsing(bench, tmp_path):
    """The clocks entry of the report: the median SM clock over the samples
    taken under load (utilisation >= 50 %), the maximum clock, and every
    throttle reason seen active (nvidia-smi CSV rows, no header, no units)."""
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join([
        "0, 345, 2070, 120.5, 0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 900.1, 100, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1380.0, 100, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.2, 99, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc, s.path = Done(), str(path)
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    assert not path.exists()
