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

  value  inferences/s with the query's inputs already in HBM (device pointers),
         the server path of a batch of one replayed as a CUDA graph
         (value_eager: the same with every kernel launched on the stream);
  e2e    the same through helrm_infer_e2e from pinned host buffers, the
         host->device copy of the query and the device->host read of the
         logit inside the timed region.
The default line also carries "batched": 16 UCI-shaped queries of 8 clients
through one lockstep batch (helrm_infer_batch_e2e_device), against the same
16 queries one at a time.

--workload criteo   the same line for the Criteo-shaped DLRM (one query/step).
--workload uci_silu the UCI-shaped line with polynomial activations: every
                    activation a degree-6 SiLU polynomial (depth 4, 18 of
                    the 20 levels, no bootstrapping).
--workload batched  64 concurrent queries per step, 32 UCI-shaped (16 clients)
                    and 32 Criteo-shaped (8 clients), each model's queries in
                    one lockstep batch; keys truncated to the levels each
                    model uses them at (helrm_model_keygen).
--workload served   the request loop (helrm_server_run) on Poisson traces,
                    80% UCI / 20% Criteo, 32 + 8 clients with resident keys:
                    p50/p99 latency and inferences/s per arrival rate, for
                    the continuous-batching server and for the plain
                    one-request-at-a-time path.
Multi-GPU: replicas (each rank its own clients and queries, no collective);
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
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 100 for the one-query workloads, 20 for batched and --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uci", choices=["uci", "criteo", "uci_silu", "batched", "served"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=1000, help="served: requests per arrival rate")
    ap.add_argument("--rates", default="1,5,10,20,50,100,200", help="served: arrival rates (requests/s)")
    ap.add_argument("--slots", type=int, default=2, help="served: batch slots (CUDA streams) of the batching server")
    ap.add_argument("--max-batch", type=int, default=8, help="served: requests per batch of the batching server")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 100 if args.impl == "ours" and args.workload in ("uci", "criteo", "uci_silu") else 20
    return args


def workload_config(name):
    from paper_2506_18150_gb300 import synthetic as syn
    spec = {"uci": syn.uci_spec, "criteo": syn.criteo_spec, "uci_silu": syn.uci_silu_spec}[name](0)
    desc = {
        "uci": "UCI-health-shaped DLRM, 1 query/step: 10 dense, 8 tables (2..64 rows), dim 16, "
               "bottom 10-32-16, dot interaction, top 52-32-1, x^2",
        "criteo": "Criteo-shaped DLRM, 1 query/step: 13 dense, 26 tables (33.8M rows, base 64), dim 16, "
                  "bottom 13-512-256-64-16, dot interaction, top 367-512-256-1, x^2",
        "uci_silu": "UCI-health-shaped DLRM, 1 query/step, as 'uci' but every activation is a degree-6 "
                    "least-squares SiLU polynomial on [-6, 6] (depth 4, no bootstrapping; ct_dense at level 18)",
    }[name]
    cfg = {"workload": desc, "ckks": "N=2^16, q0 60-bit + 20x40-bit, K=3x60-bit special, alpha=3, Delta=2^40",
           "tables": spec.cards if name != "criteo" else f"{len(spec.cards)} tables, {sum(spec.cards)} rows",
           "l2": "no flush: each step streams ~GBs of keys and diagonals (>> 129 MB L2)"}
    return spec, cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; start()
    returns once the first sample is in (at most 5 s), so the sampling is
    live when the timed region begins."""

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
                                          "-lms", "100", "-i", str(self.idx)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
            return
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
            time.sleep(0.01)

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


# Issue-bound ceiling of the NTT: 152 SMs x 4 schedulers x 32 lanes issue at
# most 19,456 integer instructions per SM clock, and a lazy Shoup butterfly on
# 64-bit words needs at least 23 of them (three 64-bit products as 32-bit
# multiply-adds, the lazy corrections and the sum/difference).
NTT_INSTR_PER_BUTTERFLY = 23
ALU_LANES = 152 * 4 * 32


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per NTT launch
# (one transform, both passes) over the one-query UCI-shaped step, from one
# ncu capture with its default cold caches (profiles/ntt_traffic_uci_dlrm_n16.md).
# It holds for the sources it was taken on: reported while their SHA-256
# still matches, null otherwise.
NTT_TRAFFIC = {"workload": "uci", "bytes_per_launch": 19.83e6,
               "sha256": {"ntt.cu": "381430a43604fce2ae84e91c42d1e8e831cb84c3b8bb2854fe410d1d0b4a0642",
                          "core.cuh": "b07128795e4ff0ab3e8bb30502566ed472f561f9e424ae75a00afd43277c7013"}}


def ntt_traffic(workload):
    import hashlib
    if workload != NTT_TRAFFIC["workload"]:
        return None
    for name, digest in NTT_TRAFFIC["sha256"].items():
        try:
            with open(os.path.join(ROOT, "paper_2506_18150_gb300", "csrc", name), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return NTT_TRAFFIC["bytes_per_launch"]


def roofline(rep, n_steps, log_n, sm_mhz, peak_hbm, peak_src, workload=None):
    """Dominant kernel (by time) with its bound: the NTT against the issue
    ceiling (butterflies/s), everything else against measured HBM bandwidth."""
    total = sum(v[1] for v in rep.values())
    dom = max(rep, key=lambda k: rep[k][1])
    n, ms, byts = rep[dom]
    kernels = {k: {"launches_per_step": v[0] / n_steps, "ms_per_step": v[1] / n_steps,
                   "GBps": (v[2] / (v[1] / 1000.0) / 1e9) if v[1] else None}
               for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1])}
    if dom == "ntt":
        bfly = byts * log_n / 32.0                      # 16 N bytes per limb <-> (N/2) log2 N butterflies
        achieved = bfly / (ms / 1000.0) / 1e9
        peak = ALU_LANES * sm_mhz * 1e6 / NTT_INSTR_PER_BUTTERFLY / 1e9
        out = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "Gbutterfly/s",
               "frac": achieved / peak,
               "peak_source": f"derived: {ALU_LANES} lanes x {sm_mhz:.0f} MHz / {NTT_INSTR_PER_BUTTERFLY} "
                              f"instructions per butterfly",
               "hbm_GBps": byts / (ms / 1000.0) / 1e9, "hbm_frac": byts / (ms / 1000.0) / 1e9 / peak_hbm}
    else:
        achieved = byts / (ms / 1000.0) / 1e9
        out = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
               "frac": achieved / peak_hbm, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"}
    traffic = ntt_traffic(workload) if dom == "ntt" else None
    if traffic is not None:
        out["traffic_note"] = ("DRAM bytes per transform under ncu (cold caches), against "
                               f"{byts / n:.4g} algorithmic bytes per transform")
    out.update({"traffic": traffic, "launches_per_step": n / n_steps, "ms_per_step": ms / n_steps,
                "share_of_kernel_time": ms / total, "kernels": kernels})
    return out


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
    if args.workload not in ("uci", "criteo", "uci_silu"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the one-query workloads "
                          "(uci, criteo); it has no batched or served mode"}), flush=True)
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


def job_throughput(units_per_rank, ms, world, device="cuda"):
    """Whole-job throughput over replicas: the units all ranks processed over
    the slowest rank's time (an all-reduce MAX of the per-rank times when
    world > 1).  Returns (units/s, slowest ms)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1000.0), ms


def _timed(fn, reps=1):
    """CUDA-event time of reps calls of fn on the current stream, in ms per call."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def batched_probe(H, syn, ctx, model, spec, pr, n_clients=8, n_queries=16):
    """n_queries queries of n_clients clients: one lockstep batch vs one at a time."""
    import numpy as np
    import torch
    keys = [H.helrm_model_keygen(ctx, model, 4000 + c) for c in range(n_clients)]
    owner = [q % n_clients for q in range(n_queries)]
    batch = H.helrm_batch_create(ctx, model, [keys[o][1] for o in owner])
    dense, idx = syn.make_queries(spec, n_queries, seed=4100)
    dd = torch.tensor(dense, dtype=torch.float64, device="cuda")
    di = torch.tensor(idx.astype(np.int64), dtype=torch.int64, device="cuda")
    lb = torch.zeros(n_queries, dtype=torch.float64, device="cuda")
    ls = torch.zeros(n_queries, dtype=torch.float64, device="cuda")

    def one_at_a_time():
        for q in range(n_queries):
            sk, evk = keys[owner[q]]
            H.helrm_infer_e2e_device(ctx, sk, evk, model, dd[q].data_ptr(), di[q].data_ptr(), 1, 11 + 2 * q,
                                     ls[q:q + 1].data_ptr())

    def lockstep():
        H.helrm_infer_batch_e2e_device(ctx, batch, [keys[o][0] for o in owner], dd.data_ptr(), di.data_ptr(), 11,
                                       lb.data_ptr())
    one_at_a_time()
    lockstep()
    torch.cuda.synchronize()
    t1 = _timed(one_at_a_time, 2)
    tb = _timed(lockstep, 2)
    return {"queries": n_queries, "clients": n_clients, "keys": "helrm_model_keygen (truncated per level)",
            "value": n_queries / (tb / 1000.0), "one_at_a_time": n_queries / (t1 / 1000.0),
            "speedup": t1 / tb, "same_logits": bool(torch.equal(lb, ls)), "unit": UNIT}


def run_batched(args):
    """Config 4: 64 concurrent queries per step (32 UCI-shaped of 16 clients,
    32 Criteo-shaped of 8 clients), each model's queries one lockstep batch."""
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
    groups = []
    for name, spec_fn, n_cl, n_q in [("uci", syn.uci_spec, 16, 32), ("criteo", syn.criteo_spec, 8, 32)]:
        spec = spec_fn(0)
        model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
        keys = [H.helrm_model_keygen(ctx, model, 10_000 * (rank + 1) + 100 * len(groups) + c) for c in range(n_cl)]
        owner = [q % n_cl for q in range(n_q)]
        batch = H.helrm_batch_create(ctx, model, [keys[o][1] for o in owner])
        K, W = args.steps, args.warmup
        dense, idx = syn.make_queries(spec, n_q * (K + W), seed=600 + rank * 10 + len(groups))
        groups.append(dict(name=name, spec=spec, model=model, keys=keys, owner=owner, batch=batch, n_q=n_q,
                           dense=dense, idx=idx, nd=dense.shape[1], nt=idx.shape[1],
                           d_dense=torch.tensor(dense, dtype=torch.float64, device="cuda"),
                           d_idx=torch.tensor(idx.astype(np.int64), dtype=torch.int64, device="cuda"),
                           d_lg=torch.zeros(n_q * (K + W), dtype=torch.float64, device="cuda")))
    K, W = args.steps, args.warmup
    n_step = sum(g["n_q"] for g in groups)

    def step(s):
        for g in groups:
            o = s * g["n_q"]
            H.helrm_infer_batch_e2e_device(ctx, g["batch"], [g["keys"][x][0] for x in g["owner"]],
                                           g["d_dense"][o].data_ptr(), g["d_idx"][o].data_ptr(), 21 + 2 * o,
                                           g["d_lg"][o:].data_ptr())

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for s in range(W):
        step(s)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = H.helrm_ctx_launch_count(ctx)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record(stream)
    for s in range(K):
        step(W + s)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    launches = H.helrm_ctx_launch_count(ctx) - l0
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(K))
    value, total_ms = job_throughput(n_step * K, ev[0].elapsed_time(ev[K]), world)

    # e2e: each step's inputs copied from pinned host memory, logits read back
    host = [(torch.from_numpy(np.ascontiguousarray(g["dense"])).pin_memory(),
             torch.from_numpy(np.ascontiguousarray(g["idx"].astype(np.uint64)).view(np.int64)).pin_memory(),
             torch.zeros(g["d_lg"].numel(), dtype=torch.float64).pin_memory()) for g in groups]

    def step_e2e(s):
        for g, (hd, hi, hl) in zip(groups, host):
            o = s * g["n_q"]
            g["d_dense"][o:o + g["n_q"]].copy_(hd[o:o + g["n_q"]], non_blocking=True)
            g["d_idx"][o:o + g["n_q"]].copy_(hi[o:o + g["n_q"]], non_blocking=True)
        step(s)
        for g, (hd, hi, hl) in zip(groups, host):
            o = s * g["n_q"]
            hl[o:o + g["n_q"]].copy_(g["d_lg"][o:o + g["n_q"]], non_blocking=True)
    barrier()
    e2e_value, e2e_ms = job_throughput(n_step, _timed(lambda: [step_e2e(W + s) for s in range(K)]) / K, world)
    same = all(torch.equal(hl[W * g["n_q"]:], g["d_lg"][W * g["n_q"]:].cpu()) for g, (_, _, hl) in zip(groups, host))

    # the plain one-request-at-a-time path on the same 64 queries
    def plain(s):
        for g in groups:
            for q in range(g["n_q"]):
                o = s * g["n_q"] + q
                sk, evk = g["keys"][g["owner"][q]]
                H.helrm_infer_e2e_device(ctx, sk, evk, g["model"], g["d_dense"][o].data_ptr(),
                                         g["d_idx"][o].data_ptr(), 1, 21 + 2 * o, g["d_lg"][o:o + 1].data_ptr())
    plain_ms = _timed(lambda: plain(W))
    plain_value = n_step / (plain_ms / 1000.0)
    plain_same = all(torch.equal(host[i][2][W * g["n_q"]:(W + 1) * g["n_q"]],
                                 g["d_lg"][W * g["n_q"]:(W + 1) * g["n_q"]].cpu()) for i, g in enumerate(groups))

    H.helrm_ctx_profile(ctx, True)
    step(W)
    rep = H.helrm_ctx_profile_report(ctx)
    H.helrm_ctx_profile(ctx, False)
    peak, peak_src = peaks()
    roof = roofline(rep, 1, pr["log_n"], clk.get("sm_mhz") or 2070.0, peak, peak_src)
    mem = H.helrm_ctx_memory_in_use(ctx)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u64", "data": "synthetic (seeded; shapes of the paper's UCI/Criteo workloads)",
                "config": {"workload": "batched: 64 concurrent encrypted queries per step, 32 UCI-shaped "
                                       "(16 clients) + 32 Criteo-shaped (8 clients), one lockstep batch per model",
                           "ckks": "N=2^16, q0 60-bit + 20x40-bit, K=3x60-bit special, alpha=3, Delta=2^40",
                           "keys": "per client, each key truncated to the levels its model uses it at",
                           "device_bytes_held": mem, "parallelism": f"replicas x{world}",
                           "l2": "no flush: each step streams tens of GB of keys (>> 129 MB L2)"},
                "latency_ms": {"p50_step": per[len(per) // 2], "max_step": per[-1]},
                "clocks": clk, "gpu_launches": int(launches),
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": sum(8 * g["n_q"] * (g["nd"] + g["nt"]) for g in groups),
                        "d2h_bytes_per_step": 8 * n_step, "same_logits_as_value_path": bool(same)},
                "one_at_a_time": {"value": plain_value, "unit": UNIT, "same_logits": bool(plain_same),
                                  "speedup_of_batched": value / plain_value},
                "roofline": roof}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_served(args):
    """Config 5: Poisson arrivals, 80% UCI / 20% Criteo, 32 + 8 clients with
    resident keys; the continuous-batching server vs the plain path."""
    import numpy as np
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pr = syn.PARAMS["full"]
    ctx = H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"],
                             device=local, stream=torch.cuda.current_stream().cuda_stream)
    specs = [syn.uci_spec(0), syn.criteo_spec(0)]
    models = [H.helrm_model_create(ctx, s, syn.make_weights(s, 0)) for s in specs]
    n_uci, n_crit = 32, 8
    cmodel = [0] * n_uci + [1] * n_crit
    keys = [H.helrm_model_keygen(ctx, models[m], 20_000 * (rank + 1) + c) for c, m in enumerate(cmodel)]
    key_bytes = sum(H.helrm_evk_bytes(ctx, k[1]) for k in keys)
    servers = {"batched": H.helrm_server_create(ctx, args.slots, args.max_batch, 0),
               "one_at_a_time": H.helrm_server_create(ctx, 1, 1, 0)}
    for srv in servers.values():
        for c, m in enumerate(cmodel):
            H.helrm_server_add_client(ctx, srv, models[m], keys[c][1])
    rates = [float(x) for x in args.rates.split(",")]
    results = []
    clocks = ClockSampler(local)
    clocks.start()
    l0 = H.helrm_ctx_launch_count(ctx)
    for rate in rates:
        arrival, client = syn.serving_trace(rate, args.requests, n_uci, n_crit, 0.8, seed=int(rate * 10) + rank)
        pools = [syn.make_queries(specs[m], int(np.sum(np.array([cmodel[c] for c in client]) == m)) or 1,
                                  seed=700 + m + int(rate)) for m in range(2)]
        used = [0, 0]
        cts = []
        for r in range(len(arrival)):
            c = int(client[r])
            m = cmodel[c]
            dense, idx = pools[m][0][used[m]], pools[m][1][used[m]]
            used[m] += 1
            cts.append(H.helrm_encrypt_query(ctx, keys[c][1], models[m], dense, idx, 3 * r + 1))
        torch.cuda.synchronize()
        row = {"rate_per_s": rate, "requests": len(arrival)}
        firsts = {}
        for name, srv in servers.items():
            outs, lat, st = H.helrm_server_run(ctx, srv, arrival, client, [x[0] for x in cts], [x[1] for x in cts])
            firsts[name] = [H.helrm_ct_export(ctx, outs[r])[0] for r in range(min(16, len(outs)))]
            del outs
            row[name] = {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                         "inferences_per_s": st["throughput"], "makespan_s": st["makespan_s"],
                         "batches": st["n_batches"], "mean_batch": st["mean_batch"], "max_batch": st["max_batch"],
                         "max_inflight": st["max_inflight"]}
        row["same_logits_sampled"] = all(np.array_equal(a, b) for a, b in zip(firsts["batched"],
                                                                             firsts["one_at_a_time"]))
        del cts
        results.append(row)
    clk = clocks.stop()
    launches = H.helrm_ctx_launch_count(ctx) - l0
    top = results[-1]
    if rank == 0:
        line = {"metric": METRIC, "value": top["batched"]["inferences_per_s"], "unit": UNIT, "n_gpus": world,
                "steps": len(rates), "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64",
                "data": "synthetic (seeded Poisson traces; shapes of the paper's UCI/Criteo workloads)",
                "config": {"workload": f"served: Poisson arrivals at {args.rates} requests/s, {args.requests} "
                                       "requests per rate, 80% UCI-shaped / 20% Criteo-shaped, 32 + 8 clients",
                           "server": f"{args.slots} batch slots (CUDA streams), up to {args.max_batch} requests "
                                     "of one model per batch",
                           "baseline_server": "1 slot, 1 request per batch (the plain path)",
                           "resident_key_bytes": key_bytes, "parallelism": f"replicas x{world}"},
                "value_note": "inferences/s of the batching server at the highest arrival rate",
                "latency_ms": {"p50": top["batched"]["p50_ms"], "p99": top["batched"]["p99_ms"]},
                "clocks": clk, "gpu_launches": int(launches), "rates": results}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


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

    # the same query through a batch of one whose server path is replayed as a
    # CUDA graph (helrm_batch_set_graph; bit-identical to the eager path): the
    # client's packing and encryption and the decryption stay eager
    bt1 = H.helrm_batch_create(ctx, model, [evk])
    H.helrm_batch_set_graph(ctx, bt1, True)

    def step_graph(q):
        H.helrm_infer_batch_e2e_device(ctx, bt1, [sk], d_dense[q].data_ptr(), d_idx[q].data_ptr(), 7 + 2 * q,
                                       d_logit[q:q + 1].data_ptr())

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- value_eager: inputs resident in HBM, every kernel launched on the stream
    for q in range(W):
        step_dev(q)
    barrier()
    l0 = H.helrm_ctx_launch_count(ctx)
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ee[0].record(stream)
    for s in range(K):
        step_dev(W + s)
    ee[1].record(stream)
    barrier()
    launches_per_step = (H.helrm_ctx_launch_count(ctx) - l0) / K   # the graph replays the same kernels
    value_eager, _ = job_throughput(K, ee[0].elapsed_time(ee[1]), world)

    # ---- value: the same steps with the server path replayed as a graph
    for q in range(W):
        step_graph(q)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    clocks = ClockSampler(local)
    clocks.start()
    ncu_range = os.environ.get("HELRM_PROFILE_RANGE") == "1"   # lets `ncu --profile-from-start off` see only these steps
    if ncu_range:
        torch.cuda.profiler.start()
    ev[0].record(stream)
    for s in range(K):
        step_graph(W + s)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if ncu_range:
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    barrier()
    launches = launches_per_step * K
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    value, total_ms = job_throughput(K, ev[0].elapsed_time(ev[K]), world)
    logits = d_logit.cpu().numpy()

    # ---- e2e: pinned host buffers through helrm_infer_e2e
    h_dense = torch.from_numpy(np.ascontiguousarray(dense)).pin_memory()
    h_idx = torch.from_numpy(np.ascontiguousarray(idx.astype(np.uint64)).view(np.int64)).pin_memory()
    h_out = torch.zeros(K + W, dtype=torch.float64).pin_memory()
    L = H.lib()
    dp = ctypes.POINTER(ctypes.c_double)
    up = ctypes.POINTER(ctypes.c_uint64)

    sks = (ctypes.c_void_p * 1)(sk.ptr.value)

    def step_host(q):   # helrm_infer_batch_e2e: the graph-replayed batch of one, host buffers
        st = L.helrm_infer_batch_e2e(ctx.ptr, bt1.ptr, sks, ctypes.c_void_p(h_dense.data_ptr() + 8 * nd * q),
                                     ctypes.c_void_p(h_idx.data_ptr() + 8 * nt * q), 7 + 2 * q,
                                     ctypes.c_void_p(h_out.data_ptr() + 8 * q))
        if st != 0:
            raise H.HelrmError(st, L.helrm_last_error(ctx.ptr).decode())

    def step_host_eager(q):   # helrm_infer_e2e: every kernel launched on the stream, host buffers
        st = L.helrm_infer_e2e(ctx.ptr, sk.ptr, evk.ptr, model.ptr,
                               ctypes.cast(h_dense.data_ptr() + 8 * nd * q, dp),
                               ctypes.cast(h_idx.data_ptr() + 8 * nt * q, up), 1, 7 + 2 * q,
                               ctypes.cast(h_out.data_ptr() + 8 * q, dp), None)
        if st != 0:
            raise H.HelrmError(st, L.helrm_last_error(ctx.ptr).decode())

    def timed_host(fn):
        for q in range(W):
            fn(q)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(K):
            fn(W + s)
        e1.record(stream)
        torch.cuda.synchronize()
        return job_throughput(K, e0.elapsed_time(e1), world)[0]

    e2e_eager = timed_host(step_host_eager)
    e2e_value = timed_host(step_host)
    same = bool(np.allclose(h_out.numpy()[W:], logits[W:], atol=1e-9))

    # ---- kernel roofline: per-kernel CUDA events on the launch stream
    H.helrm_ctx_profile(ctx, True)
    n_prof = min(K, 5)
    for s in range(n_prof):
        step_dev(W + s)
    rep = H.helrm_ctx_profile_report(ctx)
    H.helrm_ctx_profile(ctx, False)
    peak, peak_src = peaks()
    roof = roofline(rep, n_prof, pr["log_n"], clk.get("sm_mhz") or 2070.0, peak, peak_src, args.workload)

    # ---- batched: 16 queries of 8 clients in one lockstep batch vs one at a time
    batched = None
    if args.workload == "uci" and world == 1:
        batched = batched_probe(H, syn, ctx, model, spec, pr)

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
                "value_eager": value_eager,
                "value_note": "value: the server path of a batch of one replayed as a CUDA graph "
                              "(helrm_infer_batch_e2e_device); value_eager: every kernel launched on the "
                              "stream (helrm_infer_e2e_device); both bit-identical",
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * (nd + nt),
                        "d2h_bytes_per_step": 8, "same_logits_as_value_path": same,
                        "api": "helrm_infer_batch_e2e (graph-replayed batch of one, host buffers)",
                        "eager": e2e_eager},
                "roofline": roof}
        if batched:
            line["batched"] = batched
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
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
