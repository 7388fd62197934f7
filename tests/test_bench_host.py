"""Host logic of bench.py that needs no GPU: the clock sampler keeps the nvidia-smi samples
taken inside the timed window (by their timestamps), else the nearest one, flagged."""
from __future__ import annotations

import datetime
import importlib.util
import os
import pathlib
import tempfile

ROOT = pathlib.Path(__file__).resolve().parents[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _sampler(rows):
    b = _bench()
    c = b.ClockSampler(0)
    fd, c.path = tempfile.mkstemp()
    os.close(fd)
    with open(c.path, "w") as f:
        for t, mhz, reasons in rows:
            ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            f.write(f"{ts}, 0, {mhz}, 2070, 900.0, 0x0, " + ", ".join(reasons) + "\n")
    c.proc = _Proc()
    c.fh = open(os.devnull, "w")
    return c


NA = ["Not Active"] * 4


def test_samples_inside_window_only():
    t0 = 1.0e9
    c = _sampler([(t0 - 0.3, 900, ["Active", "Not Active", "Not Active", "Not Active"]),
                  (t0 + 0.02, 2070, NA), (t0 + 0.07, 2060, ["Not Active", "Not Active", "Not Active", "Active"]),
                  (t0 + 0.5, 1200, NA)])
    r = c.stop(t0, t0 + 0.1)
    assert r["samples"] == 2 and r["in_window"]
    assert r["sm_mhz"] == 2065.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]  # the hw_slowdown sample lies before the window


def test_nearest_sample_when_none_inside():
    t0 = 1.0e9
    c = _sampler([(t0 - 0.4, 1000, NA), (t0 + 0.15, 2050, NA)])
    r = c.stop(t0, t0 + 0.1)
    assert r["samples"] == 1 and not r["in_window"] and r["sm_mhz"] == 2050.0


def test_no_sampler():
    b = _bench()
    c = b.ClockSampler(0)
    assert c.stop(0.0, 1.0) is None
