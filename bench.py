#!/usr/bin/env python3
"""Encrypted DLRM inference on GB300: throughput, latency and kernel roofline.

One step = one encrypted DLRM inference of one query, the whole hot path:
client packing of the dense features and the digit one-hot selectors,
encoding and encryption (two ciphertexts), the server's bottom MLP, packed
embedding lookup, dot interaction and top MLP (double-hoisted BSGS matvecs,
x^2 activations), and decryption of the logit.  Default workload: the
Criteo-shaped DLRM (13 dense features, 26 tables with 33.8M rows in base 64,
dim 16, bottom 13-512-256-64-16, top 367-512-256-1), the largest one-query
configuration, at N = 2^16 with a 60-bit base prime, 20 levels of 40-bit
primes and three 60-bit special primes, synthetic seeded inputs.

  value  inferences/s with the query's inputs already in HBM (device pointers),
         the server path of a batch of one replayed as a CUDA graph
         (value_eager: the same with every kernel launched on the stream);
  e2e    the same through helrm_infer_batch_e2e from pinned host buffers: the
         host->device copy of the query's features and the device->host read
         of the logit inside the timed region (the client encrypts on the same
         GPU); e2e.server: the server's side of the protocol alone, the two
         query ciphertexts imported from host memory (helrm_ct_import), the
         inference, the logit ciphertext exported to host memory.
The default line also carries, each timed on the same GPU in the same run:
  uci      the same measurements for the UCI-shaped DLRM (10 dense, 8 tables
           of 2..64 rows, bottom 10-32-16, top 52-32-1);
  batched  16 UCI-shaped queries of 8 clients in one lockstep batch against
           the same 16 one at a time;
  config4  64 concurrent queries per step, 32 UCI-shaped (16 clients) and 32
           Criteo-shaped (8 clients), each model's queries one lockstep batch,
           against the same queries one at a time;
  served   the request loop (helrm_server_run) on Poisson traces at two
           arrival rates, 80% UCI / 20% Criteo over config4's clients, with
           p50/p99 latency, for the continuous-batching server and the plain
           one-request-at-a-time path;
  boot     bootstrapping alone (boot_measure: 512 periodic slots at N = 2^16
           on the bootstrappable chain);
  criteo_silu_boot / criteo_relu_boot   the one-query measurements of the
           Criteo-shaped model with SiLU (two bootstraps per query) and with
           a ReLU stand-in (three), on the bootstrappable chain.

--workload uci / uci_silu   the one-query line for the UCI-shaped model
                    (uci_silu: every activation a degree-6 SiLU polynomial).
--workload criteo_silu_boot / criteo_relu_boot   the one-query line for the
                    bootstrapped Criteo-shaped models.
--workload batched  config4 alone, with more steps.
--workload served   the request loop at every rate of --rates, 32 + 8 clients.
--workload tiny     config 1: one 1024 x 16 table in base 32 at N = 2^13, one
                    encrypted lookup per step (lookups/s).
--workload boot     bootstrapping alone (bootstraps/s): one bootstrap of a
                    ciphertext with 512-periodic slots per step at N = 2^16 on
                    the bootstrappable chain; the default line carries the same
                    measurement as its `boot` key.
Multi-GPU: replicas (each rank its own clients and queries, no collective);
value = all ranks' inferences / the slowest rank's time.  Without torchrun,
--gpus N > 1 starts N ranks itself.
--impl reference times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import socket
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted DLRM inferences/s"
UNIT = "inferences/s"
ONE_QUERY = ("criteo", "uci", "uci_silu", "criteo_silu_boot", "criteo_relu_boot")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 100 for the one-query workloads, 20 for --impl reference "
                         "and batched)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="criteo",
                    choices=["criteo", "uci", "uci_silu", "criteo_silu_boot", "criteo_relu_boot", "batched", "served",
                             "tiny", "boot"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="one-query line only (no uci/batched/config4/served keys)")
    ap.add_argument("--requests", type=int, default=1000, help="served: requests per arrival rate")
    ap.add_argument("--rates", default="1,5,10,20,50,100,200", help="served: arrival rates (requests/s)")
    ap.add_argument("--slots", type=int, default=2, help="served: batch slots (CUDA streams) of the batching server")
    ap.add_argument("--max-batch", type=int, default=8, help="served: requests per batch of the batching server")
    args = ap.parse_args(argv)
    if args.steps is None:
        args.steps = {"tiny": 1000}.get(args.workload, 100) if args.impl == "ours" and \
            args.workload in ONE_QUERY + ("tiny",) else 20
    return args


DESC = {
    "uci": "UCI-health-shaped DLRM, 1 query/step: 10 dense, 8 tables (2..64 rows), dim 16, "
           "bottom 10-32-16, dot interaction, top 52-32-1, x^2",
    "criteo": "Criteo-shaped DLRM, 1 query/step: 13 dense, 26 tables (33.8M rows, base 64), dim 16, "
              "bottom 13-512-256-64-16, dot interaction, top 367-512-256-1, x^2",
    "uci_silu": "UCI-health-shaped DLRM, 1 query/step, as 'uci' but every activation is a degree-6 "
                "least-squares SiLU polynomial on [-6, 6] (depth 4, no bootstrapping; ct_dense at level 18)",
    "criteo_silu_boot": "Criteo-shaped DLRM, 1 query/step, as 'criteo' but every activation is the degree-6 "
                        "SiLU polynomial (34 levels in all), with 2 bootstraps per query (before bottom layer 2, "
                        "256 slots; on z before the interaction, 512 slots)",
    "criteo_relu_boot": "Criteo-shaped DLRM, 1 query/step, as 'criteo' but every activation is a degree-14 "
                        "least-squares ReLU polynomial on [-6, 6] (44 levels in all), with 3 bootstraps per query "
                        "(before bottom layer 2, 256 slots; on z, 512 slots; before top layer 1, 512 slots)",
}
CKKS = "N=2^16, q0 60-bit + 20x40-bit, K=3x60-bit special, alpha=3, Delta=2^40"
CKKS_BOOT = "N=2^16, q0 60-bit + 13x40-bit + 13x60-bit, K=3x60-bit special, alpha=3, secret h=192, Delta=2^40"
SPECS = {"uci": "uci_spec", "criteo": "criteo_spec", "uci_silu": "uci_silu_spec",
         "criteo_silu_boot": "criteo_silu_boot_spec", "criteo_relu_boot": "criteo_relu_boot_spec"}
BOOT_WORKLOADS = ("criteo_silu_boot", "criteo_relu_boot")


def workload_config(name, world=1):
    from paper_2506_18150_gb300 import synthetic as syn
    spec = getattr(syn, SPECS[name])(0)
    cfg = {"workload": DESC[name], "ckks": CKKS_BOOT if spec.boot else CKKS,
           "tables": spec.cards if not name.startswith("criteo") else
           f"{len(spec.cards)} tables, {sum(spec.cards)} rows",
           "l2": "no flush: each step streams GBs of keys and diagonals (>> 129 MB L2)",
           "parallelism": f"replicas x{world}"}
    return spec, cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; start()
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
                                          "-lms", "50", "-i", str(self.idx)],
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


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def alu_peaks(H, ctx):
    """The integer ceilings, measured on this GPU by helrm_alu_peak: the
    register-resident rate (no memory traffic) of the NTT's forward and
    inverse lazy butterflies and of the inner products' 128-bit
    multiply-accumulates, best of 2..8 CTAs of 256 threads per SM."""
    out = {}
    for name, kind in (("fwd_butterfly", 0), ("inv_butterfly", 1), ("mac128", 2)):
        out[name] = max(H.helrm_alu_peak(ctx, kind, bps, 4096) for bps in (2, 4, 8)) / 1e9
    # the NTT runs as many forward as inverse butterflies: their mean time per butterfly
    out["ntt_butterfly"] = 2.0 / (1.0 / out["fwd_butterfly"] + 1.0 / out["inv_butterfly"])
    return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per NTT launch (one
# transform, both passes) over the one-query Criteo-shaped step, from one ncu
# capture of every NTT pass of a step with warm caches (--cache-control none,
# profiles/ntt_traffic_criteo_dlrm_n16.md), against 29.77 MB of algorithmic
# bytes per transform.  It holds for the sources it was taken on: reported
# while their SHA-256 still matches, null otherwise.
NTT_TRAFFIC = {"workload": "criteo", "bytes_per_launch": 32.80e6, "algorithmic_per_launch": 29.77e6,
               "sha256": {"ntt.cu": "3770ec2c28a75bf1784d58cd26d6dd7e72959c539994d9aa1e08ca1c465ef294",
                          "butterfly.cuh": "c18964e4e06f1b00915ec55936ad0b6bd0ad7a30966d19e64b31cc886fe0e95e",
                          "core.cuh": "9850591e1add3f99728e66f9a632545c7fecc69f2304fcd9fdc62a510748f42b"}}


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


def roofline(rep, n_steps, log_n, peak_hbm, hbm_src, alu=None, workload=None):
    """Dominant kernel (by time) with its bound: the NTT against the measured
    butterfly rate (integer issue, G butterflies/s), every other kernel
    against the measured HBM copy bandwidth."""
    total = sum(v[1] for v in rep.values())
    dom = max(rep, key=lambda k: rep[k][1])
    n, ms, byts = rep[dom]
    kernels = {k: {"launches_per_step": v[0] / n_steps, "ms_per_step": v[1] / n_steps,
                   "GBps": (v[2] / (v[1] / 1000.0) / 1e9) if v[1] else None,
                   "hbm_frac": (v[2] / (v[1] / 1000.0) / 1e9 / peak_hbm) if v[1] else None}
               for k, v in sorted(rep.items(), key=lambda kv: -kv[1][1])}
    if dom == "ntt":
        bfly = byts * log_n / 32.0                      # 16 N bytes per limb <-> (N/2) log2 N butterflies
        achieved = bfly / (ms / 1000.0) / 1e9
        if alu:
            peak, src = alu["ntt_butterfly"], ("measured: helrm_alu_peak, register-resident lazy Shoup butterflies "
                                               "(the NTT passes' code), mean of forward and inverse")
        else:
            peak, src = None, "not measured"
        out = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "Gbutterfly/s",
               "frac": achieved / peak if peak else None, "peak_source": src,
               "hbm_GBps": byts / (ms / 1000.0) / 1e9, "hbm_frac": byts / (ms / 1000.0) / 1e9 / peak_hbm}
    else:
        achieved = byts / (ms / 1000.0) / 1e9
        out = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
               "frac": achieved / peak_hbm, "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}
    traffic = ntt_traffic(workload) if dom == "ntt" else None
    if traffic is not None:
        out["traffic_note"] = ("DRAM bytes per transform (both passes) under ncu with warm caches, against "
                               f"{NTT_TRAFFIC['algorithmic_per_launch'] / 1e6:.2f} MB algorithmic per transform "
                               f"in the same capture ({byts / n / 1e6:.2f} MB in this run)")
    out.update({"traffic": traffic, "launches_per_step": n / n_steps, "ms_per_step": ms / n_steps,
                "share_of_kernel_time": ms / total, "kernels": kernels})
    if alu:
        out["alu_peaks_G_per_s"] = alu
    return out


def cpu_baseline(workload: str):
    """The oracle, as it stands, on this host's cores (subprocess: no CUDA in
    it), on a bounded sample (oracle.bench_sample --budget)."""
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    try:
        r = subprocess.run([sys.executable, "-m", "oracle.bench_sample", "--workload", workload,
                            "--budget"], cwd=ROOT, capture_output=True, text=True,
                           timeout=1200, env=env)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
    return {"value": 1.0 / d["est_full_s_per_query"], "unit": UNIT, "cores": d["cores"], "kind": "oracle",
            "sample": d["sample"]}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def spawn_replicas(n: int, script: str, argv, env=None, stdout=None) -> int:
    """Start n ranks of `script` on this node (torch.distributed.run, one
    process per GPU, rendezvous on 127.0.0.1); rank 0 prints the JSON line.
    Returns the launcher's exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), script] + list(argv)
    return subprocess.run(cmd, cwd=ROOT, env=env, stdout=stdout).returncode


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload not in ("criteo", "uci", "uci_silu"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the one-query workloads "
                          "without bootstrapping (criteo, uci, uci_silu); it has no batched or served mode, and a "
                          "bootstrap takes the oracle minutes (bench.py --workload boot reports that sample as its "
                          "cpu_baseline)"}), flush=True)
        return
    from oracle import bench_sample
    spec, cfg = workload_config(args.workload, world)
    d = bench_sample.run(args.workload, args.steps, args.warmup)
    units = d["steps_in_queries"]                 # the part of a query the timed stages cover
    value = units / (d["wall_s"] * d["ratio_to_full"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * d["wall_s"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": cfg,
            "value_note": (f"each step one stage of a query (of {d['n_stages']}) on the CPU oracle at "
                           f"N=2^{d['sample_log_n']}; the {args.steps} timed stages cover {units:.3f} queries "
                           f"(each stage weighted by its measured share of a query) in {d['wall_s']:.1f} s, "
                           f"scaled x{d['ratio_to_full']:.2f} to N=2^16 (the oracle's ring-product time ratio "
                           "measured on this host)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": d["cores"],
                             "sample": d["sample"]},
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


class Env:
    """The context and process state one run of the bench shares."""

    def __init__(self, boot_chain: bool = False):
        """boot_chain: the context on the bootstrappable chain (models with
        bootstraps), else on the 20-level chain of the other models."""
        import torch

        from paper_2506_18150_gb300 import helrm as H
        from paper_2506_18150_gb300 import synthetic as syn
        self.torch, self.H, self.syn = torch, H, syn
        self.world, self.rank, self.local = dist_env()
        torch.cuda.set_device(self.local)
        import torch.distributed as dist
        if self.world > 1 and not dist.is_initialized():
            dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
        self.stream = torch.cuda.current_stream()
        self.pr = syn.boot_params() if boot_chain else syn.PARAMS["full"]
        pr = self.pr
        self.ctx = H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"],
                                      pr["log2_scale"], device=self.local, stream=self.stream.cuda_stream)
        self.models = {}

    def model(self, name):
        if name not in self.models:
            spec = getattr(self.syn, SPECS[name])(0)
            self.models[name] = (spec, self.H.helrm_model_create(self.ctx, spec, self.syn.make_weights(spec, 0)))
        return self.models[name]

    def barrier(self):
        self.torch.cuda.synchronize()
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        self.torch.cuda.synchronize()

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def one_query(E, wl, K, W, hbm, alu, seed=1000):
    """The one-query measurements of workload wl: value (graph-replayed batch
    of one, inputs in HBM), value_eager, e2e from host features, e2e of the
    server side from host ciphertexts, per-query latency, the kernel
    roofline."""
    import ctypes

    import numpy as np
    torch, H, syn, ctx, stream = E.torch, E.H, E.syn, E.ctx, E.stream
    spec, model = E.model(wl)
    sk, evk = H.helrm_model_keygen(ctx, model, seed + E.rank)
    dense, idx = syn.make_queries(spec, K + W, seed=500 + E.rank)
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
    graph = True
    H.helrm_batch_set_graph(ctx, bt1, graph)

    def step_graph(q):
        H.helrm_infer_batch_e2e_device(ctx, bt1, [sk], d_dense[q].data_ptr(), d_idx[q].data_ptr(), 7 + 2 * q,
                                       d_logit[q:q + 1].data_ptr())

    # ---- value_eager: inputs resident in HBM, every kernel launched on the stream
    for q in range(W):
        step_dev(q)
    E.barrier()
    l0 = H.helrm_ctx_launch_count(ctx)
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ee[0].record(stream)
    for s in range(K):
        step_dev(W + s)
    ee[1].record(stream)
    E.barrier()
    launches_per_step = (H.helrm_ctx_launch_count(ctx) - l0) / K   # the graph replays the same kernels
    value_eager, _ = job_throughput(K, ee[0].elapsed_time(ee[1]), E.world)

    # ---- value: the same steps with the server path replayed as a graph
    for q in range(W):
        step_graph(q)
    E.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
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
    E.barrier()
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(K))
    value, total_ms = job_throughput(K, ev[0].elapsed_time(ev[K]), E.world)
    logits = d_logit.cpu().numpy()

    # ---- e2e: pinned host buffers through helrm_infer_batch_e2e
    h_dense = torch.from_numpy(np.ascontiguousarray(dense)).pin_memory()
    h_idx = torch.from_numpy(np.ascontiguousarray(idx.astype(np.uint64)).view(np.int64)).pin_memory()
    h_out = torch.zeros(K + W, dtype=torch.float64).pin_memory()
    L = H.lib()
    dp = ctypes.POINTER(ctypes.c_double)
    up = ctypes.POINTER(ctypes.c_uint64)
    sks = (ctypes.c_void_p * 1)(sk.ptr.value)

    def call(st):
        if st != 0:
            raise H.HelrmError(st, L.helrm_last_error(ctx.ptr).decode())

    def step_host(q):   # helrm_infer_batch_e2e: the graph-replayed batch of one, host buffers
        call(L.helrm_infer_batch_e2e(ctx.ptr, bt1.ptr, sks, ctypes.c_void_p(h_dense.data_ptr() + 8 * nd * q),
                                     ctypes.c_void_p(h_idx.data_ptr() + 8 * nt * q), 7 + 2 * q,
                                     ctypes.c_void_p(h_out.data_ptr() + 8 * q)))

    def step_host_eager(q):   # helrm_infer_e2e: every kernel launched on the stream, host buffers
        call(L.helrm_infer_e2e(ctx.ptr, sk.ptr, evk.ptr, model.ptr,
                               ctypes.cast(h_dense.data_ptr() + 8 * nd * q, dp),
                               ctypes.cast(h_idx.data_ptr() + 8 * nt * q, up), 1, 7 + 2 * q,
                               ctypes.cast(h_out.data_ptr() + 8 * q, dp), None))

    def timed_host(fn):
        for q in range(W):
            fn(q)
        E.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(K):
            fn(W + s)
        e1.record(stream)
        torch.cuda.synchronize()
        return job_throughput(K, e0.elapsed_time(e1), E.world)[0]

    e2e_eager = timed_host(step_host_eager)
    e2e_value = timed_host(step_host)
    same = bool(np.allclose(h_out.numpy()[W:], logits[W:], atol=1e-9))

    # ---- e2e of the server side: ciphertexts in from host memory, logit ciphertext out
    n_srv = min(K, 20)
    q_cts = [H.helrm_encrypt_query(ctx, evk, model, dense[q], idx[q], 7 + 2 * q) for q in range(W + n_srv)]
    if isinstance(q_cts[0][1], list):
        raise RuntimeError("server e2e expects a one-ciphertext selector")
    host_cts = []
    for cd, cs in q_cts:
        pair = []
        for ct in (cd, cs):
            coeffs, lv, sc = H.helrm_ct_export(ctx, ct)
            pair.append((torch.from_numpy(coeffs.reshape(-1).view(np.int64)).pin_memory(), lv, sc))
        host_cts.append(pair)
    del q_cts
    h2d_srv = sum(8 * t.numel() for t, _, _ in host_cts[0])
    h_logct = None

    def step_server(q):
        ins = []
        for t, lv, sc in host_cts[q]:
            o = ctypes.c_void_p()
            call(L.helrm_ct_import(ctx.ptr, ctypes.cast(t.data_ptr(), up), lv, ctypes.c_double(sc), ctypes.byref(o)))
            ins.append(H.Handle(o.value, ctx))
        y = H.helrm_infer_batch(ctx, bt1, [ins[0]], [ins[1]])[0]
        nonlocal h_logct
        if h_logct is None:   # sized once, at the first (untimed) call, for the logit's level
            h_logct = torch.zeros(2 * (H.helrm_ct_info(ctx, y)[0] + 1) << E.pr["log_n"], dtype=torch.int64)
            h_logct = h_logct.pin_memory()
        call(L.helrm_ct_export(ctx.ptr, y.ptr, ctypes.cast(h_logct.data_ptr(), up), None, None))

    for q in range(W):
        step_server(q)
    E.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(n_srv):
        step_server(W + s)
    e1.record(stream)
    torch.cuda.synchronize()
    srv_value = job_throughput(n_srv, e0.elapsed_time(e1), E.world)[0]

    # ---- kernel roofline: per-kernel CUDA events on the launch stream
    H.helrm_ctx_profile(ctx, True)
    n_prof = min(K, 5)
    for s in range(n_prof):
        step_dev(W + s)
    rep = H.helrm_ctx_profile_report(ctx)
    H.helrm_ctx_profile(ctx, False)
    roof = roofline(rep, n_prof, E.pr["log_n"], hbm[0], hbm[1], alu, wl)
    out = {"value": value, "ms_per_step": total_ms / K, "value_eager": value_eager,
           "latency_ms": {"p50": per[len(per) // 2], "p99": per[min(len(per) - 1, int(round(0.99 * (len(per) - 1))))],
                          "min": per[0], "max": per[-1]},
           "launches_per_step": launches_per_step,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * (nd + nt),
                   "d2h_bytes_per_step": 8, "same_logits_as_value_path": same,
                   "api": "helrm_infer_batch_e2e (%s batch of one, host buffers)" % ("graph-replayed" if graph
                                                                                     else "eager"),
                   "eager": e2e_eager,
                   "server": {"value": srv_value, "unit": UNIT, "steps": n_srv, "h2d_bytes_per_step": h2d_srv,
                              "d2h_bytes_per_step": 8 * h_logct.numel(),
                              "api": "helrm_ct_import x2 (query ciphertexts, coefficient domain, from pinned "
                                     "host memory) + helrm_infer_batch (%s batch of one) + "
                                     "helrm_ct_export (logit ciphertext to pinned host memory)"
                                     % ("graph-replayed" if graph else "eager")}},
           "roofline": roof}
    del bt1, sk, evk, host_cts
    gc.collect()
    return out


def batched_probe(E, n_clients=8, n_queries=16):
    """n_queries UCI-shaped queries of n_clients clients: one lockstep batch vs one at a time."""
    import numpy as np
    torch, H, syn, ctx = E.torch, E.H, E.syn, E.ctx
    spec, model = E.model("uci")
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
    out = {"queries": n_queries, "clients": n_clients, "keys": "helrm_model_keygen (truncated per level)",
           "value": n_queries / (tb / 1000.0), "one_at_a_time": n_queries / (t1 / 1000.0),
           "speedup": t1 / tb, "same_logits": bool(torch.equal(lb, ls)), "unit": UNIT}
    del batch, keys
    gc.collect()
    return out


def make_clients(E, n_uci, n_crit, seed_base):
    """Per-client keys (truncated per level) for n_uci UCI-shaped and n_crit
    Criteo-shaped clients: [(model name, sk, evk)]."""
    H, ctx = E.H, E.ctx
    out = []
    for c in range(n_uci + n_crit):
        name = "uci" if c < n_uci else "criteo"
        sk, evk = H.helrm_model_keygen(ctx, E.model(name)[1], seed_base + c)
        out.append((name, sk, evk))
    return out


def config4(E, clients, K, W, hbm, alu):
    """64 concurrent queries per step: 32 UCI-shaped (16 clients) and 32
    Criteo-shaped (8 clients), each model's queries one lockstep batch; the
    same queries one at a time."""
    import numpy as np
    torch, H, syn, ctx, stream = E.torch, E.H, E.syn, E.ctx, E.stream
    groups = []
    for name, n_q in (("uci", 32), ("criteo", 32)):
        spec, model = E.model(name)
        mine = [c for c in clients if c[0] == name]
        owner = [mine[q % len(mine)] for q in range(n_q)]
        batch = H.helrm_batch_create(ctx, model, [o[2] for o in owner])
        dense, idx = syn.make_queries(spec, n_q * (K + W), seed=600 + E.rank * 10 + len(groups))
        groups.append(dict(name=name, model=model, owner=owner, batch=batch, n_q=n_q, dense=dense, idx=idx,
                           nd=dense.shape[1], nt=idx.shape[1],
                           d_dense=torch.tensor(dense, dtype=torch.float64, device="cuda"),
                           d_idx=torch.tensor(idx.astype(np.int64), dtype=torch.int64, device="cuda"),
                           d_lg=torch.zeros(n_q * (K + W), dtype=torch.float64, device="cuda")))
    n_step = sum(g["n_q"] for g in groups)

    def step(s):
        for g in groups:
            o = s * g["n_q"]
            H.helrm_infer_batch_e2e_device(ctx, g["batch"], [x[1] for x in g["owner"]],
                                           g["d_dense"][o].data_ptr(), g["d_idx"][o].data_ptr(), 21 + 2 * o,
                                           g["d_lg"][o:].data_ptr())

    for s in range(W):
        step(s)
    E.barrier()
    l0 = H.helrm_ctx_launch_count(ctx)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record(stream)
    for s in range(K):
        step(W + s)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    E.barrier()
    launches = H.helrm_ctx_launch_count(ctx) - l0
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(K))
    value, total_ms = job_throughput(n_step * K, ev[0].elapsed_time(ev[K]), E.world)

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
    E.barrier()
    e2e_value, _ = job_throughput(n_step, _timed(lambda: [step_e2e(W + s) for s in range(K)]) / K, E.world)
    same = all(torch.equal(hl[W * g["n_q"]:], g["d_lg"][W * g["n_q"]:].cpu()) for g, (_, _, hl) in zip(groups, host))

    # the plain one-request-at-a-time path on the same 64 queries
    def plain(s):
        for g in groups:
            for q in range(g["n_q"]):
                o = s * g["n_q"] + q
                _, sk, evk = g["owner"][q]
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
    out = {"value": value, "unit": UNIT, "queries_per_step": n_step, "steps": K, "warmup": W,
           "ms_per_step": total_ms / K,
           "workload": "64 concurrent encrypted queries per step, 32 UCI-shaped (16 clients) + 32 Criteo-shaped "
                       "(8 clients), one lockstep batch per model",
           "latency_ms": {"p50_step": per[len(per) // 2], "max_step": per[-1]},
           "gpu_launches": int(launches), "device_bytes_held": H.helrm_ctx_memory_in_use(ctx),
           "e2e": {"value": e2e_value, "unit": UNIT,
                   "h2d_bytes_per_step": sum(8 * g["n_q"] * (g["nd"] + g["nt"]) for g in groups),
                   "d2h_bytes_per_step": 8 * n_step, "same_logits_as_value_path": bool(same)},
           "one_at_a_time": {"value": plain_value, "unit": UNIT, "same_logits": bool(plain_same),
                             "speedup_of_batched": value / plain_value},
           "roofline": roofline(rep, 1, E.pr["log_n"], hbm[0], hbm[1], alu)}
    for g in groups:
        g.clear()
    gc.collect()
    return out


def served(E, clients, rates, n_requests, slots, max_batch, frac_uci=0.8):
    """The request loop on Poisson traces: per rate, p50/p99 latency and
    inferences/s of the continuous-batching server and of the plain path."""
    import numpy as np
    H, syn, ctx = E.H, E.syn, E.ctx
    n_uci = sum(1 for c in clients if c[0] == "uci")
    n_crit = len(clients) - n_uci
    servers = {"batched": H.helrm_server_create(ctx, slots, max_batch, 0),
               "one_at_a_time": H.helrm_server_create(ctx, 1, 1, 0)}
    for srv in servers.values():
        for name, _, evk in clients:
            H.helrm_server_add_client(ctx, srv, E.model(name)[1], evk)
    results = []
    l0 = H.helrm_ctx_launch_count(ctx)
    for rate in rates:
        arrival, client = syn.serving_trace(rate, n_requests, n_uci, n_crit, frac_uci, seed=int(rate * 10) + E.rank)
        cmodel = [c[0] for c in clients]
        pools = {m: syn.make_queries(E.model(m)[0], int(sum(1 for c in client if cmodel[c] == m)) or 1,
                                     seed=700 + (m == "criteo") + int(rate)) for m in ("uci", "criteo")}
        used = {"uci": 0, "criteo": 0}
        cts = []
        for r in range(len(arrival)):
            c = int(client[r])
            m = cmodel[c]
            dense, idx = pools[m][0][used[m]], pools[m][1][used[m]]
            used[m] += 1
            cts.append(H.helrm_encrypt_query(ctx, clients[c][2], E.model(m)[1], dense, idx, 3 * r + 1))
        E.torch.cuda.synchronize()
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
    launches = H.helrm_ctx_launch_count(ctx) - l0
    del servers
    gc.collect()
    return {"rates": results, "gpu_launches": int(launches), "clients": f"{n_uci} UCI-shaped + {n_crit} Criteo-shaped",
            "server": f"{slots} batch slots (CUDA streams), up to {max_batch} requests of one model per batch",
            "baseline_server": "1 slot, 1 request per batch (the plain path)",
            "resident_key_bytes": sum(H.helrm_evk_bytes(ctx, c[2]) for c in clients)}


BOOT_NS = 512


def boot_measure(local, world, K, W, hbm, alu, n_s=BOOT_NS):
    """Bootstrapping (Sec. 2.1.4; the paper's Criteo models with polynomial
    activations need 12 or 5 per inference, Sec. 5.4): one bootstrap per step
    of a ciphertext whose slots repeat with period n_s (512: the widest layer
    of the Criteo-shaped model), N = 2^16 on the bootstrappable chain (q_0,
    13 x 40-bit compute primes, 13 x 60-bit bootstrapping primes, 3 special
    primes), a secret with 192 non-zero coefficients.  value: bootstraps/s
    with the input ciphertexts resident in HBM; e2e: the input ciphertext
    imported from pinned host memory, the bootstrap, the output ciphertext
    exported to pinned host memory."""
    import ctypes

    import numpy as np
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    stream = torch.cuda.current_stream()
    pr = syn.boot_params()
    ctx = H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"],
                             device=local, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    bt = H.helrm_boot_create(ctx, n_s)
    info = H.helrm_boot_info(ctx, bt)
    sk, evk = H.helrm_keygen_ex(ctx, 5, 192, H.helrm_boot_rotations(ctx, bt), conj=True)
    setup_s = time.perf_counter() - t0
    n = 1 << (pr["log_n"] - 1)
    rng = np.random.default_rng(77)
    zs = [rng.uniform(-1, 1, n_s) for _ in range(K + W)]
    cts = [H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, z[np.arange(n) % n_s], 0, 2.0**40), 3 + q)
           for q, z in enumerate(zs)]
    outs = [None] * (K + W)

    def step(q):
        outs[q] = H.helrm_bootstrap(ctx, evk, bt, cts[q])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
    for q in range(W):
        step(q)
    barrier()
    l0 = H.helrm_ctx_launch_count(ctx)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ncu_range = os.environ.get("HELRM_PROFILE_RANGE") == "1"   # lets `ncu --profile-from-start off` see only these steps
    if ncu_range:
        torch.cuda.profiler.start()
    ev[0].record(stream)
    for s in range(K):
        step(W + s)
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if ncu_range:
        torch.cuda.profiler.stop()
    launches = (H.helrm_ctx_launch_count(ctx) - l0) / K
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(K))
    value, total_ms = job_throughput(K, ev[0].elapsed_time(ev[K]), world)
    err = max(float(np.max(np.abs(H.helrm_decrypt(ctx, sk, outs[q], n_s) - zs[q]))) for q in range(W, W + K))
    for q in range(K + W):
        outs[q] = None

    # e2e: the input ciphertext from pinned host memory, the output back to it
    L = H.lib()
    up = ctypes.POINTER(ctypes.c_uint64)
    host = []
    for ct in cts:
        coeffs, lv, sc = H.helrm_ct_export(ctx, ct)
        host.append((torch.from_numpy(coeffs.reshape(-1).view(np.int64)).pin_memory(), lv, sc))
    h_out = torch.zeros(2 * (info["level_out"] + 1) << pr["log_n"], dtype=torch.int64).pin_memory()

    def call(st):
        if st != 0:
            raise H.HelrmError(st, L.helrm_last_error(ctx.ptr).decode())

    def step_e2e(q):
        t, lv, sc = host[q]
        o = ctypes.c_void_p()
        call(L.helrm_ct_import(ctx.ptr, ctypes.cast(t.data_ptr(), up), lv, ctypes.c_double(sc), ctypes.byref(o)))
        y = H.helrm_bootstrap(ctx, evk, bt, H.Handle(o.value, ctx))
        call(L.helrm_ct_export(ctx.ptr, y.ptr, ctypes.cast(h_out.data_ptr(), up), None, None))
    for q in range(W):
        step_e2e(q)
    barrier()
    e2e_value, _ = job_throughput(K, _timed(lambda: [step_e2e(W + s) for s in range(K)]), world)

    H.helrm_ctx_profile(ctx, True)
    n_prof = min(K, 3)
    for s in range(n_prof):
        step(W + s)
    rep = H.helrm_ctx_profile_report(ctx)
    H.helrm_ctx_profile(ctx, False)
    roof = roofline(rep, n_prof, pr["log_n"], hbm[0], hbm[1], alu, "boot")
    out = {"value": value, "unit": "bootstraps/s", "ms_per_step": total_ms / K,
           "latency_ms": {"p50": per[len(per) // 2], "min": per[0], "max": per[-1]},
           "launches_per_step": launches, "max_abs_err": err, "setup_s": setup_s,
           "levels": {"in": 0, "top": info["level_top"], "out": info["level_out"]},
           "e2e": {"value": e2e_value, "unit": "bootstraps/s", "h2d_bytes_per_step": 8 * host[0][0].numel(),
                   "d2h_bytes_per_step": 8 * h_out.numel(),
                   "api": "helrm_ct_import (level-0 ciphertext, pinned host memory) + helrm_bootstrap + "
                          "helrm_ct_export (refreshed ciphertext to pinned host memory)"},
           "config": {"workload": f"bootstrapping of n_s={n_s} periodic real slots, one per step (ModRaise, SubSum, "
                                  f"CoeffToSlot: one product and the conjugate of its output, EvalMod: degree-16 cosine and "
                                  f"6 double angles, SlotToCoeff)",
                      "ckks": "N=2^16, q0 60-bit + 13x40-bit + 13x60-bit, K=3x60-bit special, alpha=3, "
                              "secret h=192, Delta=2^40",
                      "l2": "no flush: each step streams GBs of keys and diagonals (>> 129 MB L2)"},
           "roofline": roof}
    del bt, sk, evk, cts, host
    gc.collect()
    del ctx
    gc.collect()
    return out


def base_line(E, args, cfg):
    return {"metric": METRIC, "unit": UNIT, "n_gpus": E.world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded; shapes of the paper's UCI/Criteo workloads)", "config": cfg}


def run_ours(args):
    E = Env(boot_chain=args.workload in BOOT_WORKLOADS)
    K, W = args.steps, args.warmup
    hbm = hbm_peak()
    alu = alu_peaks(E.H, E.ctx)
    spec, cfg = workload_config(args.workload, E.world)
    clocks = ClockSampler(E.local)
    clocks.start()
    main = one_query(E, args.workload, K, W, hbm, alu)
    extras = {}
    if args.workload == "criteo" and not args.no_extras:
        u = one_query(E, "uci", K, W, hbm, alu)
        u["config"] = workload_config("uci", E.world)[1]
        extras["uci"] = u
        if E.world == 1:
            extras["batched"] = batched_probe(E)
        clients = make_clients(E, 16, 8, 10_000 * (E.rank + 1))
        extras["config4"] = config4(E, clients, min(K, 10), min(W, 3), hbm, alu)
        extras["served"] = served(E, clients, [100.0, 200.0], 300, args.slots, args.max_batch)
        del clients
        gc.collect()
        extras["boot"] = boot_measure(E.local, E.world, min(K, 10), min(W, 3), hbm, alu)
        E2 = Env(boot_chain=True)
        for wl in BOOT_WORKLOADS:
            b = one_query(E2, wl, min(K, 10), min(W, 3), hbm, alu)
            b["config"] = workload_config(wl, E.world)[1]
            extras[wl] = b
        del E2
        gc.collect()
    clk = clocks.stop()
    if E.rank == 0:
        line = base_line(E, args, cfg)
        line.update({"value": main["value"], "ms_per_step": main["ms_per_step"], "latency_ms": main["latency_ms"],
                     "clocks": clk, "gpu_launches": int(main["launches_per_step"] * K),
                     "value_eager": main["value_eager"],
                     "value_note": "value: the server path of a batch of one replayed as a CUDA graph "
                                   "(helrm_infer_batch_e2e_device); value_eager: every kernel launched on the "
                                   "stream (helrm_infer_e2e_device); both bit-identical",
                     "e2e": main["e2e"], "roofline": main["roofline"]})
        line.update(extras)
        if E.world == 1 and not args.no_cpu_baseline and args.workload not in BOOT_WORKLOADS:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    E.close()


def run_batched(args):
    E = Env()
    K, W = args.steps, args.warmup
    hbm = hbm_peak()
    alu = alu_peaks(E.H, E.ctx)
    clients = make_clients(E, 16, 8, 10_000 * (E.rank + 1))
    clocks = ClockSampler(E.local)
    clocks.start()
    r = config4(E, clients, K, W, hbm, alu)
    clk = clocks.stop()
    if E.rank == 0:
        line = base_line(E, args, {"workload": "batched: " + r.pop("workload"), "ckks": CKKS,
                                   "keys": "per client, each key truncated to the levels its model uses it at",
                                   "parallelism": f"replicas x{E.world}",
                                   "l2": "no flush: each step streams tens of GB of keys (>> 129 MB L2)"})
        line.update({"value": r.pop("value"), "ms_per_step": r.pop("ms_per_step"), "clocks": clk,
                     "gpu_launches": r.pop("gpu_launches"), "e2e": r.pop("e2e"), "roofline": r.pop("roofline")})
        line.update(r)
        print(json.dumps(line), flush=True)
    E.close()


def run_served(args):
    E = Env()
    clients = make_clients(E, 32, 8, 20_000 * (E.rank + 1))
    rates = [float(x) for x in args.rates.split(",")]
    clocks = ClockSampler(E.local)
    clocks.start()
    r = served(E, clients, rates, args.requests, args.slots, args.max_batch)
    clk = clocks.stop()
    top = r["rates"][-1]
    if E.rank == 0:
        line = base_line(E, args, {"workload": f"served: Poisson arrivals at {args.rates} requests/s, "
                                               f"{args.requests} requests per rate, 80% UCI-shaped / 20% "
                                               "Criteo-shaped, 32 + 8 clients",
                                   "server": r["server"], "baseline_server": r["baseline_server"],
                                   "resident_key_bytes": r["resident_key_bytes"],
                                   "parallelism": f"replicas x{E.world}"})
        line.update({"value": top["batched"]["inferences_per_s"], "steps": len(rates), "warmup": 0,
                     "ms_per_step": None, "value_note": "inferences/s of the batching server at the highest "
                                                        "arrival rate",
                     "latency_ms": {"p50": top["batched"]["p50_ms"], "p99": top["batched"]["p99_ms"]},
                     "clocks": clk, "gpu_launches": r["gpu_launches"], "rates": r["rates"]})
        print(json.dumps(line), flush=True)
    E.close()


def run_boot(args):
    """--workload boot: bootstrapping alone (boot_measure), with the oracle's
    bounded CPU sample beside it."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    hbm = hbm_peak()
    pr = syn.PARAMS["full"]
    actx = H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"],
                              device=local, stream=torch.cuda.current_stream().cuda_stream)
    alu = alu_peaks(H, actx)
    del actx
    clocks = ClockSampler(local)
    clocks.start()
    r = boot_measure(local, world, args.steps, args.warmup, hbm, alu)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": "bootstraps/s", "value": r["value"], "unit": "bootstraps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic (seeded uniform slots in [-1, 1])", "config": dict(r["config"]),
                "latency_ms": r["latency_ms"], "max_abs_err": r["max_abs_err"], "levels": r["levels"],
                "clocks": clk, "gpu_launches": int(r["launches_per_step"] * args.steps), "e2e": r["e2e"],
                "roofline": r["roofline"]}
        line["config"]["parallelism"] = f"replicas x{world}"
        if world == 1 and not args.no_cpu_baseline:
            env = dict(os.environ)
            env.pop("CUDA_VISIBLE_DEVICES", None)
            try:
                p = subprocess.run([sys.executable, "-m", "oracle.bench_sample", "--workload", "boot"], cwd=ROOT,
                                   capture_output=True, text=True, timeout=900, env=env)
                d = json.loads(p.stdout.strip().splitlines()[-1])
                line["cpu_baseline"] = {"value": 1.0 / d["est_full_s_per_boot"], "unit": "bootstraps/s",
                                        "cores": d["cores"], "kind": "oracle", "sample": d["sample"]}
            except Exception as e:  # noqa: BLE001
                line["cpu_baseline"] = {"value": None, "unit": "bootstraps/s", "kind": "oracle",
                                        "sample": f"failed: {e}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_tiny(args):
    """Config 1: the 1024 x 16 table in base 32 at N = 2^13 (three 50-bit
    primes, one special prime), one encrypted lookup per step.  value:
    lookups/s of the server's lookup on selector ciphertexts already on the
    device; e2e: the client's selector (helrm_query_pack), encoding and
    encryption, the lookup and the decryption of the 16 outputs, from a host
    index to host floats, one query per step."""
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
    pr = syn.PARAMS["tiny"]
    ctx = H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"],
                             device=local, stream=stream.cuda_stream)
    delta = 2.0 ** pr["log2_scale"]
    n = 1 << (pr["log_n"] - 1)
    C = syn.tiny_table(0)
    emb = H.helrm_emb_prepare(ctx, [1024], 32, 0, 16, [C], 0, 16, 1, delta, delta)
    sk, evk = H.helrm_keygen(ctx, 0, H.helrm_ptmat_rotations(ctx, H.helrm_emb_matrix(ctx, emb, 0)))
    K, W = args.steps, args.warmup
    idx = [int(np.random.default_rng(1000 * rank + q).integers(0, 1024)) for q in range(K + W)]
    cts = [H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, H.helrm_query_pack(ctx, emb, [i], n), 1, delta), 42 + q)
           for q, i in enumerate(idx)]
    outs = [None] * (K + W)

    def step(q):
        outs[q] = H.helrm_embedding_lookup(ctx, evk, emb, cts[q])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
    for q in range(W):
        step(q)
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
    launches = H.helrm_ctx_launch_count(ctx) - l0
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(K))
    value, total_ms = job_throughput(K, ev[0].elapsed_time(ev[K]), world)
    err = max(float(np.max(np.abs(H.helrm_decrypt(ctx, sk, outs[q], 16)
                                  - (C[0][idx[q] % 32].astype(np.float64) + C[1][idx[q] // 32]))))
              for q in range(W, W + K))

    # e2e: host index in, host floats out, through the C ABI
    L = H.lib()
    out16 = np.zeros(16)

    def step_e2e(q):
        sel = H.helrm_query_pack(ctx, emb, [idx[q]], n)
        ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, sel, 1, delta), 42 + q)
        y = H.helrm_embedding_lookup(ctx, evk, emb, ct)
        st = L.helrm_decrypt(ctx.ptr, sk.ptr, y.ptr, out16.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 16)
        if st != 0:
            raise H.HelrmError(st, L.helrm_last_error(ctx.ptr).decode())
    for q in range(W):
        step_e2e(q)
    barrier()
    e2e_value, _ = job_throughput(K, _timed(lambda: [step_e2e(W + s) for s in range(K)]), world)
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": "encrypted embedding lookups/s", "value": value, "unit": "lookups/s", "n_gpus": world,
                "steps": K, "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded; the paper's tiny-table shape)",
                "config": {"workload": "tiny: one 1024 x 16 table in base 32 (2 digit one-hots of 32 slots in one "
                                       "ciphertext), one lookup per step", "ckks": "N=2^13, q 3x50-bit, P 1x50-bit, "
                                       "alpha=1, Delta=2^40", "parallelism": f"replicas x{world}",
                           "l2": "no flush: a step reads keys and diagonals once (a few MB, L2-resident)"},
                "latency_ms": {"p50": per[len(per) // 2], "max": per[-1]}, "max_abs_err": err,
                "clocks": clk, "gpu_launches": int(launches),
                "e2e": {"value": e2e_value, "unit": "lookups/s", "h2d_bytes_per_step": 8 * n,
                        "d2h_bytes_per_step": 8 * 16,
                        "api": "helrm_query_pack + helrm_encode + helrm_encrypt + helrm_embedding_lookup + "
                               "helrm_decrypt"}}
        if world == 1 and not args.no_cpu_baseline:
            env = dict(os.environ)
            env.pop("CUDA_VISIBLE_DEVICES", None)
            try:
                r = subprocess.run([sys.executable, "-m", "oracle.bench_sample", "--workload", "tiny", "--steps",
                                    "3"], cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
                d = json.loads(r.stdout.strip().splitlines()[-1])
                line["cpu_baseline"] = {"value": 1.0 / d["s_per_lookup"], "unit": "lookups/s", "cores": d["cores"],
                                        "kind": "oracle", "sample": d["sample"]}
            except Exception as e:  # noqa: BLE001
                line["cpu_baseline"] = {"value": None, "unit": "lookups/s", "kind": "oracle", "sample": f"failed: {e}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "0"))
    if args.gpus > 1 and not world:
        sys.exit(spawn_replicas(args.gpus, os.path.abspath(__file__), sys.argv[1:]))
    if world and args.gpus != world:
        sys.exit(f"--gpus {args.gpus} does not match WORLD_SIZE {world}")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "tiny":
        run_tiny(args)
    elif args.workload == "boot":
        run_boot(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
