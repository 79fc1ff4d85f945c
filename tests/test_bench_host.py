"""Host logic of bench.py, on CPU: the roofline arithmetic (the NTT against
its measured integer ceiling, any other kernel against the HBM peak), the
parsing of nvidia-smi clock samples with their throttle reasons, and the
oracle arm's accounting of stage samples."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_ntt_against_measured_ceiling():
    # 89 transforms moving 1190 MB (algorithmic) in 2.29 ms, per step
    rep = {"ntt": (89, 2.29, 1190e6), "bsgs_fused": (5, 1.27, 3.8e9)}
    alu = {"fwd_butterfly": 800.0, "inv_butterfly": 800.0, "mac128": 3600.0, "ntt_butterfly": 800.0}
    r = bench.roofline(rep, 1, 16, 6787.6, "measured", alu)
    assert r["bound"] == "alu" and r["kernel"] == "ntt" and r["unit"] == "Gbutterfly/s"
    # 16 N bytes per limb <-> (N/2) log2 N butterflies: bytes * 16 / 32 butterflies
    assert abs(r["achieved"] - 1190e6 * 16 / 32 / 2.29e-3 / 1e9) < 1e-9
    assert r["peak"] == 800.0 and abs(r["frac"] - r["achieved"] / 800.0) < 1e-12
    assert r["peak_source"].startswith("measured")
    assert abs(r["hbm_frac"] - 1190e6 / 2.29e-3 / 1e9 / 6787.6) < 1e-12
    assert r["launches_per_step"] == 89 and abs(r["share_of_kernel_time"] - 2.29 / 3.56) < 1e-12
    # without a measured ceiling there is no fraction
    r = bench.roofline(rep, 1, 16, 6787.6, "measured", None)
    assert r["peak"] is None and r["frac"] is None


def test_roofline_hbm_bound_kernel():
    rep = {"ntt": (10, 0.5, 100e6), "bsgs_fused": (5, 1.0, 3.4e9)}
    r = bench.roofline(rep, 2, 16, 6800.0, "fallback")
    assert r["bound"] == "hbm" and r["kernel"] == "bsgs_fused" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 3.4e9 / 1e-3 / 1e9) < 1e-6 and abs(r["frac"] - 3400.0 / 6800.0) < 1e-12
    assert r["traffic"] is None and r["launches_per_step"] == 2.5
    assert abs(r["kernels"]["ntt"]["hbm_frac"] - 100e6 / 0.5e-3 / 1e9 / 6800.0) < 1e-12


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


def test_stage_records_give_query_time():
    from oracle import bench_sample
    recs = [(0, 0, 1.0), (0, 1, 3.0), (0, 2, 2.0), (1, 0, 1.2), (1, 1, 2.8)]
    assert abs(bench_sample.query_time(recs, 3) - (1.1 + 2.9 + 2.0)) < 1e-12
    for k, v in bench_sample.STAGE_SHARES.items():
        assert abs(sum(v) - 1.0) < 2e-3, k


def test_parse_defaults():
    a = bench.parse([])
    assert a.workload == "criteo" and a.gpus == 1 and a.steps == 100 and a.warmup == 3
    a = bench.parse(["--impl", "reference", "--steps", "20", "--warmup", "5"])
    assert a.steps == 20 and a.warmup == 5


def test_ntt_traffic_follows_the_measured_sources(monkeypatch):
    assert bench.ntt_traffic("criteo") == bench.NTT_TRAFFIC["bytes_per_launch"]
    assert bench.ntt_traffic("uci") is None                 # measured on the Criteo-shaped step only
    changed = dict(bench.NTT_TRAFFIC, sha256=dict(bench.NTT_TRAFFIC["sha256"], **{"ntt.cu": "0" * 64}))
    monkeypatch.setattr(bench, "NTT_TRAFFIC", changed)
    assert bench.ntt_traffic("criteo") is None              # the kernel changed since the capture
    r = bench.roofline({"ntt": (145, 6.35, 4.5e9)}, 1, 16, 6787.6, "measured", None, "criteo")
    assert r["traffic"] is None
