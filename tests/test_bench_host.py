"""Host logic of bench.py: the FP32 peak it reports against, the clock sampler's parsing of the
nvidia-smi record (throttle reasons decide whether a run is kept) and the percentile helper."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_fp32_alu_peak():
    # 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz
    assert bench.fp32_alu_peak_tflops(152, 2070) == pytest.approx(80.54784, rel=1e-12)


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler_with(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(line + "\n" for line in lines))
    s = bench.ClockSampler(0)
    s.proc = _DoneProcess()
    s.path = str(path)
    return s


def test_clock_sampler_median_max_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 912.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1380.25, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    ]
    r = _sampler_with(tmp_path, rows).stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_clock_sampler_reports_every_slowdown(tmp_path):
    rows = [
        "0, 1500, 2070, 700.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, 1400, 2070, 650.0, 0x0000000000000040, Not Active, Active, Active, Not Active",
        "garbled line",
    ]
    r = _sampler_with(tmp_path, rows).stop()
    assert r["samples"] == 2
    assert r["sm_mhz"] == 1450.0
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_samples(tmp_path):
    r = _sampler_with(tmp_path, []).stop()
    assert r["samples"] == 0 and r["sm_mhz"] is None and r["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)            # nvidia-smi never started
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_percentile():
    a = list(range(1, 101))
    assert bench.percentile(a, 50) == pytest.approx(50.5)
    assert bench.percentile(a, 99) == pytest.approx(99.01)
