"""Host logic of bench.py, on CPU: the roofline arithmetic (the NTT against
its integer-issue ceiling, any other kernel against the HBM peak), the guard
that reports the measured NTT traffic only while the sources it was measured
on are unchanged, and the parsing of nvidia-smi clock samples with their
throttle reasons."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_ntt_against_issue_ceiling():
    # 89 transforms moving 1190 MB (algorithmic) in 2.29 ms, per step
    rep = {"ntt": (89, 2.29, 1190e6), "bsgs_fused": (5, 1.27, 3.8e9)}
    r = bench.roofline(rep, 1, 16, 2070.0, 6787.6, "measured", "criteo")
    assert r["bound"] == "alu" and r["kernel"] == "ntt" and r["unit"] == "Gbutterfly/s"
    # 16 N bytes per limb <-> (N/2) log2 N butterflies: bytes * 16 / 32 butterflies
    assert abs(r["achieved"] - 1190e6 * 16 / 32 / 2.29e-3 / 1e9) < 1e-9
    assert abs(r["peak"] - 152 * 4 * 32 * 2070e6 / 23 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["traffic"] is None                       # measured for the UCI step only
    assert r["launches_per_step"] == 89 and abs(r["share_of_kernel_time"] - 2.29 / 3.56) < 1e-12


def test_roofline_hbm_bound_kernel():
    rep = {"ntt": (10, 0.5, 100e6), "bsgs_fused": (5, 1.0, 3.4e9)}
    r = bench.roofline(rep, 2, 16, 2070.0, 6800.0, "fallback", "uci")
    assert r["bound"] == "hbm" and r["kernel"] == "bsgs_fused" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 3.4e9 / 1e-3 / 1e9) < 1e-6 and abs(r["frac"] - 3400.0 / 6800.0) < 1e-12
    assert r["traffic"] is None and r["launches_per_step"] == 2.5


def test_ntt_traffic_follows_the_measured_sources(monkeypatch):
    assert bench.ntt_traffic("uci") == bench.NTT_TRAFFIC["bytes_per_launch"]
    assert bench.ntt_traffic("criteo") is None
    changed = dict(bench.NTT_TRAFFIC, sha256=dict(bench.NTT_TRAFFIC["sha256"], **{"ntt.cu": "0" * 64}))
    monkeypatch.setattr(bench, "NTT_TRAFFIC", changed)
    assert bench.ntt_traffic("uci") is None           # the kernel changed since the capture
    r = bench.roofline({"ntt": (89, 2.29, 1190e6)}, 1, 16, 2070.0, 6787.6, "measured", "uci")
    assert r["traffic"] is None


def test_clock_samples_and_reasons():
    s = bench.ClockSampler(0)
    s.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    s.t = type("T", (), {"join": lambda self, timeout=None: None})()
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s.lines = ["0, 1500, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active"]
    assert s.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.stop()["samples"] == 0
