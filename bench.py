#!/usr/bin/env python3
"""Encrypted DLRM inference on GB300: throughput, latency and kernel roofline.

One step = one encrypted DLRM inference of one query, the whole hot path:
client packing of the dense features and the digit one-hot selectors,
encoding and encryption (two ciphertexts), the server's bottom MLP, packed
embedding lookup, dot interaction and top MLP (double-hoisted BSGS matvecs,
x^2 activations), and decryption of the logit.  Default workload: the
UCI-health-shaped DLRM (10 dense features, 8 tables of 2..64 rows, dim 16,
bottom 10-32-16, top 52-32-1) at N = 2^16 with a 60-bit base prime, 20
levels of 40-bit primes and three 60-bit special primes, synthetic seeded
inputs.

  value  inferences/s with the query's inputs already in HBM (device pointers);
  e2e    the same through helrm_infer_e2e from pinned host buffers, the
         host->device copy of the query and the device->host read of the
         logit inside the timed region.
Multi-GPU: replicas (each rank its own client and queries, no collective);
value = all ranks' inferences / the slowest rank's time.
--impl reference times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted DLRM inferences/s"
UNIT = "inferences/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uci", choices=["uci", "criteo"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_config(name):
    from paper_2506_18150_gb300 import synthetic as syn
    spec = syn.uci_spec(0) if name == "uci" else syn.criteo_spec(0)
    desc = {
        "uci": "UCI-health-shaped DLRM, 1 query/step: 10 dense, 8 tables (2..64 rows), dim 16, "
               "bottom 10-32-16, dot interaction, top 52-32-1, x^2",
        "criteo": "Criteo-shaped DLRM, 1 query/step: 13 dense, 26 tables (33.8M rows, base 64), dim 16, "
                  "bottom 13-512-256-64-16, dot interaction, top 367-512-256-1, x^2",
    }[name]
    cfg = {"workload": desc, "ckks": "N=2^16, q0 60-bit + 20x40-bit, K=3x60-bit special, alpha=3, Delta=2^40",
           "tables": spec.cards if name == "uci" else f"{len(spec.cards)} tables, {sum(spec.cards)} rows",
           "l2": "no flush: each step streams ~GBs of keys and diagonals (>> 129 MB L2)"}
    return spec, cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(workload: str):
    """The oracle, as it stands, on this host's cores (subprocess: no CUDA in it)."""
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    try:
        r = subprocess.run([sys.executable, "-m", "oracle.bench_sample", "--workload", workload,
                            "--steps", "2", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True,
                           timeout=900, env=env)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
    return {"value": 1.0 / d["est_full_s_per_query"], "unit": UNIT, "cores": d["cores"], "kind": "oracle",
            "sample": (f"2 queries of the same model at N=2^{d['sample_log_n']} (same levels, keys, limbs per op), "
                       f"median {d['sample_s_per_query']:.2f} s, scaled x{d['ratio_to_full']:.2f} "
                       f"(measured oracle ring-product time ratio N=2^16 : N=2^{d['sample_log_n']})")}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import bench_sample
    spec, cfg = workload_config(args.workload)
    d = bench_sample.run(args.workload, args.steps, args.warmup)
    per = [t * d["ratio_to_full"] for t in d["sample_times_s"]]
    total = sum(per)
    value = len(per) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(per),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": d["cores"],
                             "sample": f"each step one query at N=2^{d['sample_log_n']} scaled x"
                                       f"{d['ratio_to_full']:.2f} to N=2^16"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import ctypes

    import numpy as np
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    pr = syn.PARAMS["full"]
    ctx = H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"],
                             device=local, stream=stream.cuda_stream)
    spec, cfg = workload_config(args.workload)
    w = syn.make_weights(spec, 0)
    model = H.helrm_model_create(ctx, spec, w)
    sk, evk = H.helrm_keygen(ctx, 1000 + rank, H.helrm_model_rotations(ctx, model))
    K, W = args.steps, args.warmup
    dense, idx = syn.make_queries(spec, K + W, seed=500 + rank)
    d_dense = torch.tensor(dense, dtype=torch.float64, device="cuda")
    d_idx = torch.tensor(idx.astype(np.int64), dtype=torch.int64, device="cuda")
    d_logit = torch.zeros(K + W, dtype=torch.float64, device="cuda")
    nd, nt = dense.shape[1], idx.shape[1]

    def step_dev(q):
        H.helrm_infer_e2e_device(ctx, sk, evk, model, d_dense[q].data_ptr(), d_idx[q].data_ptr(), 1,
                                 7 + 2 * q, d_logit[q:q + 1].data_ptr())

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- value: inputs resident in HBM
    for q in range(W):
        step_dev(q)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    l0 = H.helrm_ctx_launch_count(ctx)
    clocks = ClockSampler(local)
    clocks.start()
    ncu_range = os.environ.get("HELRM_PROFILE_RANGE") == "1"   # lets `ncu --profile-from-start off` see only these steps
    if ncu_range:
        torch.cuda.profiler.start()
    ev[0].record(stream)
    for s in range(K):
        step_dev(W + s)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if ncu_range:
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    barrier()
    launches = H.helrm_ctx_launch_count(ctx) - l0
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    total_ms = ev[0].elapsed_time(ev[K])
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * K / (total_ms / 1000.0)
    logits = d_logit.cpu().numpy()

    # ---- e2e: pinned host buffers through helrm_infer_e2e
    h_dense = torch.from_numpy(np.ascontiguousarray(dense)).pin_memory()
    h_idx = torch.from_numpy(np.ascontiguousarray(idx.astype(np.uint64)).view(np.int64)).pin_memory()
    h_out = torch.zeros(K + W, dtype=torch.float64).pin_memory()
    L = H.lib()
    dp = ctypes.POINTER(ctypes.c_double)
    up = ctypes.POINTER(ctypes.c_uint64)

    def step_host(q):
        st = L.helrm_infer_e2e(ctx.ptr, sk.ptr, evk.ptr, model.ptr,
                               ctypes.cast(h_dense.data_ptr() + 8 * nd * q, dp),
                               ctypes.cast(h_idx.data_ptr() + 8 * nt * q, up), 1, 7 + 2 * q,
                               ctypes.cast(h_out.data_ptr() + 8 * q, dp), None)
        if st != 0:
            raise H.HelrmError(st, L.helrm_last_error(ctx.ptr).decode())

    for q in range(W):
        step_host(q)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(K):
        step_host(W + s)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = world * K / (e2e_ms / 1000.0)
    same = bool(np.allclose(h_out.numpy()[W:], logits[W:], atol=1e-9))

    # ---- kernel roofline: per-kernel CUDA events on the launch stream
    H.helrm_ctx_profile(ctx, True)
    n_prof = min(K, 5)
    for s in range(n_prof):
        step_dev(W + s)
    rep = H.helrm_ctx_profile_report(ctx)
    H.helrm_ctx_profile(ctx, False)
    prof_total = sum(v[1] for v in rep.values())
    dom = max(rep, key=lambda k: rep[k][1])
    n, ms, byts = rep[dom]
    peak, peak_src = peaks()
    achieved = byts / (ms / 1000.0) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": None, "launches_per_step": n / n_prof, "ms_per_step": ms / n_prof,
            "share_of_kernel_time": ms / prof_total,
            "kernels": {k: {"launches_per_step": v[0] / n_prof, "ms_per_step": v[1] / n_prof,
                            "GBps": (v[2] / (v[1] / 1000.0) / 1e9) if v[1] else None}
                        for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1])}}

    if rank == 0:
        per_sorted = sorted(per)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u64", "data": "synthetic (seeded; shapes of the paper's UCI/Criteo workloads)",
                "config": dict(cfg, parallelism=f"replicas x{world}"),
                "latency_ms": {"p50": per_sorted[len(per) // 2],
                               "p99": per_sorted[min(len(per) - 1, int(round(0.99 * (len(per) - 1))))],
                               "min": per_sorted[0], "max": per_sorted[-1]},
                "clocks": clk, "gpu_launches": int(launches),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * (nd + nt),
                        "d2h_bytes_per_step": 8, "same_logits_as_value_path": same},
                "roofline": roof}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
