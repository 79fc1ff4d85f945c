"""CPU timing of the oracle for bench.py (test infrastructure only).

The oracle runs the encrypted DLRM exactly as the library does (same model,
same levels, same rotations, same number of limbs per operation) but on a
reduced ring degree, because one full-size query plus its keys would take
minutes on the host.  Every per-operation cost scales with N only, so the
full-size time is estimated as

    t_full = t_sample * r,   r = t(polymul, N_full) / t(polymul, N_sample),

with r measured on the same host (ring products dominate the oracle's time).
Usage: python -m oracle.bench_sample --workload uci --steps 3 --warmup 1
prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import ckks, dlrm, ring


def _params(log_n: int, levels: int):
    return ckks.Params(log_n, [60] + [40] * levels, 3, 60, 3, 40.0)


def polymul_ratio(log_full: int, log_sample: int, limbs: int = 8, reps: int = 3) -> float:
    def t(log_n):
        p = _params(log_n, limbs - 1)
        rng = np.random.default_rng(0)
        a = np.stack([rng.integers(0, q, p.N, dtype=np.uint64) for q in p.q])
        best = 1e9
        for _ in range(reps):
            t0 = time.perf_counter()
            ckks.polymul(p, a, a, p.q)
            best = min(best, time.perf_counter() - t0)
        return best
    return t(log_full) / t(log_sample)


def run(workload: str = "uci", steps: int = 3, warmup: int = 1):
    from paper_2506_18150_gb300 import synthetic as syn
    spec = {"uci": syn.uci_spec, "criteo": syn.criteo_spec, "uci_silu": syn.uci_silu_spec}[workload](0)
    w = syn.make_weights(spec, 0)
    log_sample = 15 if workload == "criteo" else 13
    n_bot, n_top = len(w.bottom_W), len(w.top_W)
    ad = dlrm.activation_levels(spec)
    levels = (1 + ad) * (n_top - 1) + 1 + 2 + (1 + ad) * n_bot     # dot interaction
    p = _params(log_sample, levels)
    t0 = time.perf_counter()
    c = dlrm.compile_model(p, spec, w)
    sk, keys = ckks.keygen(p, 1, rot_steps=c.rotation_steps())
    setup = time.perf_counter() - t0
    dense, idx = syn.make_queries(spec, steps + warmup, seed=500)
    times = []
    for q in range(steps + warmup):
        t0 = time.perf_counter()
        cd, cs = dlrm.encrypt_query(p, keys, c, dense[q], idx[q], 100 + 2 * q)
        out = dlrm.infer(p, keys, c, cd, cs)
        dlrm.decrypt_logit(p, sk, out)
        if q >= warmup:
            times.append(time.perf_counter() - t0)
    r = polymul_ratio(16, log_sample)
    t_sample = float(np.median(times))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {
        "workload": workload,
        "sample_log_n": log_sample,
        "sample_s_per_query": t_sample,
        "sample_times_s": times,
        "ratio_to_full": r,
        "est_full_s_per_query": t_sample * r,
        "setup_s": setup,
        "cores": cores,
    }


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="uci")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args()
    print(json.dumps(run(a.workload, a.steps, a.warmup)))
