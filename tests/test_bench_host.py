"""Host-side pieces of bench.py on CPU: the clock record taken during the timed region
(median SM clock, the throttle reasons that were active, malformed or missing samples),
the pair count of the Ginteractions metric, and the whole-job rate."""
import bench
import workloads as W


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return "0, %s, %s, 900.00, 0x0000000000000000, %s, %s, %s, %s" % (sm, mx, hw, hwt, swt, pcap)


def test_clock_summary_reports_the_median_and_the_active_reasons():
    c = bench.ClockSampler(0)
    c.lines = [_line(2070, 2070), _line(2055, 2070, pcap="Active"), _line(2070, 2070),
               "garbage", "", _line("[N/A]", 2070), _line(1995, 2070, hwt="Active")]
    s = c.summary()
    assert s["sm_mhz"] == 2062.5                       # median of 2070, 2055, 2070, 1995
    assert s["sm_max_mhz"] == 2070.0
    assert s["samples"] == 4
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples_says_so():
    c = bench.ClockSampler(0)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_pair_count_is_the_sum_over_bodies_of_own_times_other_nodes():
    wl = W.two_spheres()
    assert bench.interbody_pairs(wl) == 2 * 4100 * 4100
    wl = W.spheroids8()
    n = 32320
    assert bench.interbody_pairs(wl) == 8 * n * 7 * n == 58496614400


def test_whole_job_rate_counts_every_ranks_solves():
    assert bench.whole_job_rate(3, 1, 1, 3000.0) == 1.0
    assert bench.whole_job_rate(3, 16, 4, 2000.0) == 3 * 16 * 4 / 2.0
