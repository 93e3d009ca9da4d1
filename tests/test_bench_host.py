"""Host-side pieces of bench.py on CPU: the clock record taken during the
timed region, the ring matching behind the accuracy columns, and the seeds
that keep replicas' frames disjoint."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

# nvidia-smi --format=csv,noheader,nounits rows of the sampler's fields:
# index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
_ROWS = """0, 1965, 2070, 812.4, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 1980, 2070, 903.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, [N/A], 2070, 905.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 1995, 2070, 899.9, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
truncated line
"""


def _sampler_on(tmp_path, text):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write(text)
    s.proc = subprocess.Popen([sys.executable, "-c", "import time; time.sleep(30)"])
    return s


def test_clock_record(tmp_path):
    out = _sampler_on(tmp_path, _ROWS).stop()
    assert out["samples"] == 4                      # the truncated line is dropped
    assert out["sm_mhz"] == 1980.0                  # median of the numeric samples
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]       # "Not Active" is not "Active"
    assert not os.path.exists(str(tmp_path / "clocks.csv"))


def test_clock_record_flags_thermal(tmp_path):
    rows = "0, 1500, 2070, 1390.0, 0x48, Active, Not Active, Active, Not Active\n"
    out = _sampler_on(tmp_path, rows).stop()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_no_sampler_gives_empty_record():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = None
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_accuracy_matching():
    truth = np.array([[100.0, 100.0, 20.0], [300.0, 200.0, 40.0], [500.0, 500.0, 10.0]])
    rings = np.zeros(3, dtype=[("cx", "<f4"), ("cy", "<f4"), ("r", "<f4")])
    rings["cx"] = [100.25, 301.0, 900.0]
    rings["cy"] = [99.5, 200.0, 900.0]
    rings["r"] = [20.0, 40.5, 10.0]
    acc = bench._accuracy(rings, truth)
    assert acc["recall"] == pytest.approx(2 / 3)
    assert acc["median_abs_cx_px"] == pytest.approx(0.625)
    assert acc["median_abs_cy_px"] == pytest.approx(0.25)
    assert acc["median_abs_r_px"] == pytest.approx(0.25)
    found = np.array([[300.5, 200.0, 40.0], [100.0, 101.0, 20.5]])
    assert bench._match(truth, found).tolist() == [1, 0, -1]


def test_replica_seeds_are_disjoint():
    from paper_1310_1371_gb300.replicas import frame_seeds
    seen = set()
    for rank in range(8):
        s = {tuple(x) for x in frame_seeds(rank, 96)}
        assert len(s) == 96 and not (s & seen)
        seen |= s
