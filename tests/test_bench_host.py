"""Host logic of bench.py that decides what its JSON line reports about the
clocks: nvidia-smi CSV lines (the FIELDS order of ClockSampler) summarised
into the median SM clock, the maximum clock and the throttle reasons seen
Active.  No GPU and no nvidia-smi needed."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _line(sm, mx, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", power="Not Active"):
    return f"0, {sm} MHz, {mx} MHz, 912.40 W, 0x0000000000000004, {hw}, {thermal}, {sw_thermal}, {power}\n"


def test_clean_run(bench):
    s = bench.ClockSampler.summarise([_line(2070, 2070)] * 4 + [_line(1965, 2070)])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_reasons_are_collected_by_name(bench):
    lines = [_line(2070, 2070), _line(1800, 2070, power="Active"), _line(1700, 2070, hw="Active"),
             _line(1650, 2070, thermal="Active", sw_thermal="Active")]
    s = bench.ClockSampler.summarise(lines)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == pytest.approx((1800 + 1700) / 2) and s["samples"] == 4


def test_unparsable_lines_are_skipped(bench):
    lines = ["", "garbage\n", "0, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n",
             "0, 2070 MHz, 2070 MHz\n", _line(1500, 2070)]
    s = bench.ClockSampler.summarise(lines)
    assert s == {"sm_mhz": 1500.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 1}
    assert bench.ClockSampler.summarise(lines[:4]) is None


def test_sampler_without_nvidia_smi_reports_nothing(bench, tmp_path, monkeypatch):
    """Where nvidia-smi cannot be started the sampler records nothing and
    leaves no file behind."""
    monkeypatch.setenv("PATH", str(tmp_path))
    monkeypatch.delenv("HEGET_CLOCKS_CSV", raising=False)
    c = bench.ClockSampler()
    c.start()
    assert c.proc is None and c.stop() is None and not os.path.exists(c.path)
