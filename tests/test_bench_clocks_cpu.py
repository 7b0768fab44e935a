"""bench.py's clock record (no GPU): the samples of the timed region are summarised, a
short region with none inside takes the warm-up samples just before it, and throttle
reasons are read from their columns."""
import bench


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, {hwt}, {swt}, {pcap}"


def _sampler(samples):
    c = bench.ClockSampler(0)
    c.lines = list(samples)
    return c


def test_samples_inside_the_timed_region():
    c = _sampler([(0.0, _line(345, 2070)), (10.0, _line(2070, 2070)), (10.1, _line(2055, 2070)),
                  (10.2, _line(2070, 2070, pcap="Active")), (20.0, _line(345, 2070))])
    s = c.summary(9.95, 10.25)
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_short_region_takes_the_warm_up_samples_before_it():
    # idle samples long before, one under load 0.1 s before the region, none inside
    c = _sampler([(0.0, _line(345, 2070)), (9.9, _line(2070, 2070)), (11.0, _line(345, 2070))])
    s = c.summary(10.0, 10.05)
    assert s["samples"] == 1 and s["sm_mhz"] == 2070.0


def test_throttle_reasons_and_no_samples():
    c = _sampler([(1.0, _line(1500, 2070, hw="Active", swt="Active"))])
    s = c.summary(0.5, 1.5)
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _sampler([]).summary(0.0, 1.0)["reasons"] == ["unavailable"]
