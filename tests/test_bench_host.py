"""Host-side helpers of bench.py, on CPU: the clock record keeps only the
samples taken inside the timed window and reports every throttle reason seen
there; the sysfs CPU list of the GPU's PCI device is parsed as the kernel
writes it."""
import datetime

import bench


def _line(t0, dt_ms, sm, reasons=()):
    ts = (t0 + datetime.timedelta(milliseconds=dt_ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ", ".join("Active" if n in reasons else "Not Active" for n in names)
    return f"{ts}, 0, {sm}, 2070, 900.0, 0x0, {flags}"


def test_clock_summary_keeps_the_timed_window():
    t0 = datetime.datetime.now().replace(microsecond=0)
    c = bench.ClockSampler(0)
    c.lines = [_line(t0, 0, 1200), _line(t0, 50, 2070), _line(t0, 100, 2055, ("sw_power_cap",)),
               _line(t0, 150, 2070), _line(t0, 200, 900, ("hw_slowdown",))]
    c.mark(t0.timestamp() + 0.04, t0.timestamp() + 0.16)
    s = c.summary()
    assert s["samples"] == 3 and s["sampled"] == "timed region"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]          # the slowdown after the window is not counted
    assert abs(s["window_ms"] - 120.0) < 1e-6


def test_clock_summary_short_window_and_no_samples():
    t0 = datetime.datetime.now().replace(microsecond=0)
    c = bench.ClockSampler(0)
    c.lines = [_line(t0, 0, 2070), _line(t0, 50, 2070, ("hw_thermal_slowdown",))]
    c.mark(t0.timestamp() + 0.01, t0.timestamp() + 0.02)   # between two samples
    s = c.summary()
    assert s["samples"] == 2 and s["sampled"] == "warm-up and timed region"
    assert s["reasons"] == ["hw_thermal_slowdown"]
    c.lines = ["not a sample", ""]
    assert c.summary()["reasons"] == ["unsampled"]


def test_parse_cpulist():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


def test_local_fp64_issue_view():
    # two solves of the 2048^2 headline's size: (nnz(B) + 6 K) x iterations
    # FP64 instructions over the event time
    per = [{"K": 160000, "nnzB": 800000, "it_local": 240}, {"K": 160000, "nnzB": 800000, "it_local": 240}]
    v = bench.local_fp64_issue(per, 3.6e-3)
    dp = 2 * (800000 + 6 * 160000) * 240
    assert abs(v["achieved"] - dp / 3.6e-3 / 1e9) < 1e-9
    assert v["bound"] == "alu" and abs(v["frac"] - v["achieved"] / (152 * 2 * 2.07)) < 1e-12
    assert bench.local_fp64_issue(per, 0.0)["achieved"] == 0.0
