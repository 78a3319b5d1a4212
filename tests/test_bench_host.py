"""Host-side pieces of bench.py without a GPU: the clock sampler keeps only samples taken inside
the timed region (falling back to the nearest ones for a region shorter than its period) and
reports throttle reasons; the JSON config is the workload alone, the same in both arms."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def _sampler(lines, t0, t1):
    c = bench.Clocks(0)
    c.lines = lines
    c.proc, c.t = _Proc(), _Thread()
    c.t0, c.t1 = c._when(t0), c._when(t1)
    return c.stop()


def _line(stamp, sm, cap="Not Active", thermal="Not Active"):
    return "%s, 0, %d, 2032, 900.0, 0x0, Not Active, %s, Not Active, %s" % (stamp, sm, thermal, cap)


def test_samples_inside_the_timed_region_only():
    lines = [_line("2026/12/04 05:00:00.950", 1100),  # warm-up, before the region
             _line("2026/12/04 05:00:01.010", 2032, cap="Active"),
             _line("2026/12/04 05:00:01.030", 2032),
             _line("2026/12/04 05:00:01.050", 2016),
             _line("2026/12/04 05:00:01.200", 900, thermal="Active")]  # after the region
    r = _sampler(lines, "2026/12/04 05:00:01.000", "2026/12/04 05:00:01.060")
    assert r["samples"] == 3 and r["window"] == "timed region"
    assert r["sm_mhz"] == 2032.0 and r["reasons"] == ["sw_power_cap"]


def test_short_region_takes_the_nearest_samples():
    lines = [_line("2026/12/04 05:00:00.500", 2032), _line("2026/12/04 05:00:01.100", 2032),
             _line("2026/12/04 05:00:03.000", 1000)]
    r = _sampler(lines, "2026/12/04 05:00:01.000", "2026/12/04 05:00:01.005")
    assert r["samples"] == 2 and r["window"].startswith("nearest")
    assert r["sm_mhz"] == 2032.0


def test_config_is_the_workload_alone():
    from paper_2203_08395_b300 import synth as S

    wl = S.config("layered10k")
    c = bench.workload_config("layered10k", wl)
    assert c["workload"] == "layered10k" and c["tasks"] == wl.n_tasks and c["edges"] == wl.n_edges
    assert set(c) == {"workload", "tasks", "edges", "graphs", "saxpy_elems", "l2"}


def test_small_workloads_are_timed_after_an_l2_flush():
    from types import SimpleNamespace

    small = SimpleNamespace(n_tasks=10_000, n_edges=24_000, saxpy_elems=0, graphs=[None])
    large = SimpleNamespace(n_tasks=10_000_000, n_edges=35_000_000, saxpy_elems=0, graphs=[None] * 256)
    assert bench.l2_flush_needed(small) and not bench.l2_flush_needed(large)
    assert bench.FLUSH_BYTES >= 2 * bench.L2_BYTES
    assert bench.workload_config("s", small)["l2"].startswith("L2 flushed before every timed step")
    assert bench.workload_config("l", large)["l2"].startswith("inputs larger than L2")
