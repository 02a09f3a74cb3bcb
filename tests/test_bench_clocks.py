"""Host logic of bench.py's clock sampler: only samples taken inside the timed
region count, and an active slowdown reason is reported (no GPU needed)."""
import datetime
import importlib.util
import os
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Stopped:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _sampler_with(tmp_path, rows):
    """A ClockSampler whose nvidia-smi output is the given rows:
    (seconds from now, sm MHz, power-cap state, thermal state)."""
    b = _bench()
    s = b.ClockSampler.__new__(b.ClockSampler)
    s.path = str(tmp_path / "clocks.csv")
    now = time.time()
    with open(s.path, "w") as f:
        for dt, mhz, cap, thermal in rows:
            stamp = datetime.datetime.fromtimestamp(now + dt).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            f.write(f"{stamp}, {mhz}, 2032, 700.0, 0x0, Not Active, Not Active, {thermal}, {cap}\n")
    s.proc = _Stopped()
    s.f = open(str(tmp_path / "unused"), "w")
    return s, now


def test_only_samples_inside_the_timed_region_count(tmp_path):
    s, now = _sampler_with(tmp_path, [(-2.0, 900, "Not Active", "Not Active"),
                                      (0.01, 2032, "Not Active", "Not Active"),
                                      (0.06, 2010, "Not Active", "Not Active"),
                                      (0.11, 2032, "Not Active", "Not Active"),
                                      (1.5, 900, "Active", "Active")])
    c = s.stop(now, now + 0.1)
    assert c["samples"] == 3 and c["window"] == "timed region"
    assert c["sm_mhz"] == 2032.0 and c["sm_max_mhz"] == 2032.0
    assert c["reasons"] == []


def test_reasons_inside_the_region_are_reported(tmp_path):
    s, now = _sampler_with(tmp_path, [(0.02, 1800, "Active", "Not Active"),
                                      (0.07, 1500, "Not Active", "Active")])
    c = s.stop(now, now + 0.1)
    assert c["samples"] == 2
    assert c["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]


def test_no_sample_inside_falls_back_to_the_whole_run(tmp_path):
    s, now = _sampler_with(tmp_path, [(-3.0, 2032, "Not Active", "Not Active"),
                                      (3.0, 2032, "Not Active", "Not Active")])
    c = s.stop(now, now + 0.1)
    assert c["samples"] == 2 and c["window"].startswith("whole run")
