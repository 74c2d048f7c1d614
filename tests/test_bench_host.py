"""Host logic of bench.py that needs no GPU: the clock sampler's summary of
nvidia-smi rows (median SM clock and throttle reasons over the samples whose
gpu_idle reason is not active, so that idle samples before the timed region
do not count)."""
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _summary(rows, t0=None, t1=None):
    import bench
    cs = bench.ClockSampler("0")
    cs.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    cs.fh.write("".join(r + "\n" for r in rows))
    cs.fh.flush()
    cs.proc = _Done()
    return cs.stop(t0, t1)


TS = "2026/12/04 16:18:24.000, "
IDLE = TS + "2070, 2070, 180.5, 0x1, Not Active, Not Active, Not Active, Not Active, Active"


def test_idle_samples_before_the_load_are_left_out():
    s = _summary([IDLE, IDLE,
                  TS + "1650, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active, Not Active",
                  TS + "1710, 2070, 1385.0, 0x4, Not Active, Not Active, Not Active, Active, Not Active",
                  TS + "1690, 2070, 1388.0, 0x4, Not Active, Not Active, Not Active, Active, Not Active"])
    assert s["samples"] == 3 and s["samples_total"] == 5
    assert s["sm_mhz"] == 1690.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_throttle_reasons_of_loaded_samples_are_reported():
    s = _summary([TS + "1500, 2070, 1300.0, 0x20, Not Active, Active, Not Active, Not Active, Not Active",
                  TS + "1600, 2070, 1310.0, 0x4, Not Active, Not Active, Not Active, Active, Not Active"])
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1550.0


def test_all_idle_keeps_every_sample():
    s = _summary([IDLE, IDLE])
    assert s["samples"] == 2 and s["sm_mhz"] == 2070.0


def test_rows_without_power_keep_every_sample_and_bad_rows_are_skipped():
    s = _summary([TS + "1800, 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active, Not Active",
                  "garbage",
                  TS + "1900, 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active, Not Active"])
    assert s["samples"] == 2 and s["power_w_median"] is None
    assert s["sm_mhz"] == 1850.0


def test_no_rows_give_no_summary():
    assert _summary([]) is None


def test_samples_outside_the_timed_region_are_left_out():
    import datetime
    def row(sec, mhz):
        return ("2026/12/04 16:18:%06.3f, %d, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active, "
                "Not Active" % (sec, mhz))
    t0 = datetime.datetime(2026, 12, 4, 16, 18, 10).timestamp()
    t1 = datetime.datetime(2026, 12, 4, 16, 18, 11).timestamp()
    s = _summary([row(9.5, 2070), row(10.2, 1600), row(10.7, 1640), row(11.5, 2070)], t0, t1)
    assert s["samples"] == 2 and s["sm_mhz"] == 1620.0
