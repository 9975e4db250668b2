"""bench.py's measurement helpers on the CPU: the DRAM-traffic figure of a
kernel is reported only while the kernel's source and the shared arithmetic
header are unchanged since the ncu capture, and the clock record is built
from the nvidia-smi samples inside the timed window."""
import datetime as dt
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSRC = os.path.join("paper_2305_15116_gb300", "csrc")


def _tree(tmp_path, entry_source="interior2d.cu"):
    """A copy of the two hashed sources and the committed traffic records."""
    os.makedirs(tmp_path / CSRC)
    for f in (entry_source, "arith.cuh"):
        shutil.copy(os.path.join(ROOT, CSRC, f), tmp_path / CSRC / f)
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(ROOT, "profiles", "ncu_traffic.json"), tmp_path / "profiles" / "ncu_traffic.json")
    return tmp_path


def test_traffic_only_while_the_sources_are_unchanged(tmp_path, monkeypatch):
    key = "k_interior2d_f64_square32jit_L11"
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        recorded = json.load(f)[key]
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic(key) == recorded["dram_bytes_per_launch"]
    assert recorded["dram_bytes_per_launch"] == recorded["dram_read_bytes"] + recorded["dram_write_bytes"]
    assert bench.ncu_traffic("k_no_such_kernel") is None
    # any change of the kernel's source, or of the arithmetic header it
    # includes, withdraws the figure
    for f in ("interior2d.cu", "arith.cuh"):
        p = root / CSRC / f
        keep = p.read_bytes()
        p.write_bytes(keep + b"\n")
        assert bench.ncu_traffic(key) is None, f
        p.write_bytes(keep)
        assert bench.ncu_traffic(key) == recorded["dram_bytes_per_launch"]


def _row(t, sm, mx=2070, reasons=("Not Active",) * 4):
    ts = dt.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return [ts, str(sm), str(mx), "900.0", "0x0"] + list(reasons)


def test_clock_summary_takes_the_samples_of_the_timed_window():
    t0 = 1_700_000_000.0
    rows = [_row(t0 - 1.0, 1000)] + [_row(t0 + 0.05 * i, 2070) for i in range(11)] + [_row(t0 + 5.0, 900)]
    out = bench.ClockSampler.summarise(rows, t0, t0 + 0.5)
    assert out["samples"] == 11 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and "note" not in out


def test_clock_summary_names_throttle_reasons():
    t0 = 1_700_000_000.0
    active = ("Not Active", "Active", "Not Active", "Active")  # hw_thermal_slowdown, sw_power_cap
    rows = [_row(t0 + 0.1, 1500, reasons=active), _row(t0 + 0.2, 2070)]
    out = bench.ClockSampler.summarise(rows, t0, t0 + 0.3)
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == (1500.0 + 2070.0) / 2


def test_clock_summary_of_a_window_shorter_than_the_sampling_period():
    t0 = 1_700_000_000.0
    rows = [_row(t0 - 0.4, 1980), _row(t0 + 0.3, 2070)]
    out = bench.ClockSampler.summarise(rows, t0, t0 + 0.01)
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0 and "note" in out
    assert bench.ClockSampler.summarise([], t0, t0 + 1.0)["samples"] == 0
