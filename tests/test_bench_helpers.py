"""CPU checks of the measurement arithmetic in bench.py: the unit count of a
coarse step, the roofline fraction, and when the captured DRAM traffic is
reported (only for the kernel sources it was captured on, only when every
timed launch ran the kernel it was captured for)."""
import numpy as np

import bench


def test_cell_updates_count_every_substep():
    # levels 2, 3, 4 under lmin 2: 1, 2 and 4 advances per coarse step
    leaves = np.array([(0, 0, 2, 0, 0), (0, 0, 3, 2, 0), (0, 0, 4, 8, 0)], dtype=np.int32)
    assert bench.cell_updates(leaves, 2, 32) == (1 + 2 + 4) * 32 * 32


def test_roofline_of_is_bytes_over_time():
    r = bench.roofline_of((2.0, 10, 4.0e9), 6760.6, "measured")
    assert r["achieved"] == 2000.0           # 4 GB in 2 ms
    assert abs(r["frac"] - 2000.0 / 6760.6) < 1e-15
    assert r["avg_launch_us"] == 200.0 and r["bytes_per_launch"] == 4.0e8
    assert r["traffic"] is None and r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_measured_traffic_follows_the_captured_sources(monkeypatch):
    per_patch = (36 * 36 + 32 * 32) * 4.0
    phase = (1.0, 4, 4 * 50 * per_patch)     # 4 launches of 50 patches each
    band = {0: {"variant": "band"}, 5: {"variant": "band"}}
    monkeypatch.setitem(bench.KERNEL_SOURCES_SHA, "band", bench.sources_sha("band"))
    t = bench.measured_traffic(phase, band, 4, 32)
    assert abs(t - bench.DRAM_PER_PATCH[("band", 4, 32)] * 50) < 1e-6
    assert bench.measured_traffic(phase, {"all": {"variant": "band"}}, 4, 32) == t
    mixed = {0: {"variant": "band"}, 5: {"variant": "walk"}}
    assert bench.measured_traffic(phase, mixed, 4, 32) is None
    assert bench.measured_traffic(phase, {0: {"variant": "walk"}}, 4, 32) is None
    assert bench.measured_traffic(phase, band, 8, 32) is None    # no capture for FP64
    monkeypatch.setitem(bench.KERNEL_SOURCES_SHA, "band", "0" * 16)
    assert bench.measured_traffic(phase, band, 4, 32) is None   # sources changed since

