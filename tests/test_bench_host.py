"""Host-side pieces of the benchmark (CPU): the clock sampler's summary
(throttle reasons that invalidate a run, median SM clock), the traffic record
lookup (only valid for the current assembly-kernel sources) and the
single-rank aggregation."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(rows, t0=0.0, times=None):
    c = bench.ClockSampler(0)
    c.t0 = t0
    times = times or [1.0] * len(rows)
    c.rows = [[t] + [p.strip() for p in r.split(",")] for t, r in zip(times, rows)]
    return c.summary()


def test_clock_summary_reasons_and_median():
    s = _sampler(["2070, 2070, 800.5, Not Active, Not Active, Not Active, Not Active",
                  "2055, 2070, 900.0, Not Active, Not Active, Not Active, Active",
                  "2070, 2070, 950.0, Not Active, Not Active, Not Active, Not Active"])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    s = _sampler(["1500, 2070, 700, Active, Not Active, Active, Not Active"])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s = _sampler(["[N/A], [N/A], [N/A], Not Active, Not Active, Not Active, Not Active"])
    assert s["sm_mhz"] is None and s["reasons"] == []


def test_clock_summary_uses_the_timed_region():
    """Samples taken before the timed region began (sampler start-up, idle
    clocks) are left out when the region has samples of its own."""
    rows = ["1200, 2070, 200, Not Active, Not Active, Not Active, Not Active",
            "2070, 2070, 900, Not Active, Not Active, Not Active, Not Active",
            "2070, 2070, 950, Not Active, Not Active, Not Active, Active"]
    s = _sampler(rows, t0=10.0, times=[9.0, 10.5, 10.6])
    assert s["samples"] == 2 and s["sm_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    s = _sampler(rows[:1], t0=10.0, times=[9.0])        # region shorter than one period
    assert s["samples"] == 1 and s["sm_mhz"] == 1200.0


def test_clock_summary_unsampled():
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_traffic_record_tracks_kernel_sources():
    h = bench.kernel_hash()
    assert len(h) == 16
    recs = {}
    for line in open(bench.TRAFFIC_FILE):
        if line.startswith("workload="):
            rec = dict(kv.split("=", 1) for kv in line.split())
            recs[rec["workload"]] = rec
    assert {"tri4m", "tet5m"} <= set(recs)
    for w, rec in recs.items():
        t = bench.measured_traffic(w)
        if rec.get("kernel_hash") == h:
            assert t == float(rec["dram_bytes_per_launch"])
        else:
            assert t is None                      # stale record: reported as null
    assert bench.measured_traffic("no-such-workload") is None


def test_single_rank_aggregate():
    assert bench.aggregate(12.5, 1e6, 1) == (12.5, 1e6)
