"""Host-side logic of bench.py that needs no GPU: the clock sampler's parsing
and timed-region filter, and the whole-job totals of a single process."""
import os
import sys
import time

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))

import bench  # noqa: E402


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _stamp(t):
    return time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(t)) + ".%03d" % int((t % 1) * 1000)


def _clocks_with(tmp_path, rows, window):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        for t, mhz, power_cap in rows:
            f.write(f"{_stamp(t)}, 0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, "
                    f"{'Active' if power_cap else 'Not Active'}\n")
    c.proc = _DoneProc()
    if window:
        c.mark(*window)
    return c.stop()


def test_clock_samples_outside_the_timed_region_are_dropped(tmp_path):
    t0 = time.time()
    out = _clocks_with(tmp_path, [(t0 - 1.0, 900, True), (t0 + 0.010, 2070, False), (t0 + 0.040, 2050, False),
                                  (t0 + 0.500, 1200, True)], (t0, t0 + 0.05))
    assert out["samples"] == 2 and out["sm_mhz"] == 2060.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []


def test_short_region_keeps_the_first_sample_after_it_began(tmp_path):
    t0 = time.time()
    out = _clocks_with(tmp_path, [(t0 - 0.5, 1000, False), (t0 + 0.2, 2070, True), (t0 + 0.4, 2070, False)],
                       (t0, t0 + 0.01))
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"]


def test_without_a_window_every_sample_counts(tmp_path):
    t0 = time.time()
    out = _clocks_with(tmp_path, [(t0, 2000, False), (t0 + 0.1, 2070, False)], None)
    assert out["samples"] == 2 and out["sm_mhz"] == 2035.0


def test_job_totals_single_process():
    assert bench.job_totals(1.5, 1000, None, "cpu") == (1.5, 1000.0)
