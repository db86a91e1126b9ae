"""The benchmark's clock record (CPU): nvidia-smi samples taken during the timed region are
reduced to the median SM clock, the maximum clock and the throttle reasons seen, which decide
whether a run is kept.  A fake sampler process stands in for nvidia-smi."""
import importlib.util
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_clocks_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(bench, tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = _FakeProc(), str(path)
    return s


def test_median_clock_and_power_cap(bench, tmp_path):
    # fields: index, clocks.sm, clocks.max.sm, power.draw, reasons mask, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    lines = ["0, 2070, 2070, 850.12, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.50, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2055, 2070, 1201.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    r = _sampler(bench, tmp_path, lines).stop()
    assert r == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not (tmp_path / "clocks.csv").exists()


def test_every_slowdown_reason_is_reported(bench, tmp_path):
    lines = ["0, 1500, 2070, 900.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
             "0, 1400, 2070, 900.00, 0x0000000000000040, Not Active, Active, Not Active, Not Active",
             "0, 1300, 2070, 900.00, 0x0000000000000020, Not Active, Not Active, Active, Not Active",
             "malformed line"]
    r = _sampler(bench, tmp_path, lines).stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1400.0 and r["samples"] == 3


def test_no_samples_and_no_sampler(bench, tmp_path):
    r = _sampler(bench, tmp_path, []).stop()
    assert r["samples"] == 0 and r["sm_mhz"] is None and r["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)  # nvidia-smi never started
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
