"""Host logic of bench.py that runs without a GPU: the algorithmic bytes behind the roofline, the
rule that a committed DRAM-traffic figure is used only for the kernel sources it was taken on,
and the summary of the clock samples taken during the timed region."""
import json
import os

import bench


def test_algorithmic_bytes_per_site():
    # D3Q59, FP32 deviations: 58 stored populations of 4 bytes and the rest population as a float
    # pair, read once by the moments and written once by the collision (2 Q s = 472 B of the
    # metric's definition, plus the rest pair's extra 4 bytes each way)
    b = bench._algorithmic_bytes(1, 4, read_pops=False)
    # the force kernel reads the last two steps' j~ of the extrapolated u-solve start
    assert b == {"moments": 260, "force": 76, "usolve_sweep": 64, "derivs": 132, "collide": 400}
    # 16-bit storages halve the population part only
    h = bench._algorithmic_bytes(1, 2, read_pops=False)
    assert b["moments"] - h["moments"] == 58 * 2 and b["collide"] - h["collide"] == 58 * 2
    # a collision that reads the pre-collision populations (gamma != 0) moves them twice
    r = bench._algorithmic_bytes(1, 4, read_pops=True)
    assert r["collide"] - b["collide"] == 58 * 4 + 8
    # plain relaxation keeps no update vector
    assert bench._algorithmic_bytes(1, 4, False, chebyshev=False)["usolve_sweep"] == 40
    # D2Q21: 20 stored populations, 13 aux fields
    d2 = bench._algorithmic_bytes(0, 4, read_pops=False)
    assert d2["moments"] == 20 * 4 + 8 + 4 * 4 and d2["collide"] == 13 * 4 + 8 + 8 * 4 + 88


def test_traffic_is_used_only_for_the_captured_sources(tmp_path, monkeypatch):
    os.makedirs(tmp_path / "profiles")
    entry = {"dram_bytes_per_launch": 6.7e9, "sources_sha": "aaaa"}
    with open(tmp_path / "profiles" / "traffic.json", "w") as fh:
        json.dump({"spinodal3d_256": {"collide": entry}}, fh)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_sources_sha", lambda: "aaaa")
    assert bench._traffic("collide", "spinodal3d_256") == 6.7e9
    assert bench._traffic("moments", "spinodal3d_256") is None
    assert bench._traffic("collide", "droplet3d_128") is None
    monkeypatch.setattr(bench, "_kernel_sources_sha", lambda: "bbbb")  # the kernels changed since
    assert bench._traffic("collide", "spinodal3d_256") is None


def test_clock_summary():
    cs = bench.ClockSampler(0)
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    cs.samples = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
                  ["0", "1980", "2070", "1390", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
                  ["0", "2070", "2070", "1000", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["no nvidia-smi samples"]
