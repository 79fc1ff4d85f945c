"""CPU timing of the oracle for bench.py (test infrastructure only).

The oracle runs the encrypted DLRM exactly as the library does (same model,
same levels, same rotations, same number of limbs per operation) but on a
reduced ring degree, because one full-size query plus its keys takes many
minutes on the host: N = 2^13 for the UCI-shaped model, 2^15 (the smallest
degree whose slots hold its interaction layout) for the Criteo-shaped one.
Every per-operation cost scales with N only, so a full-size time is
estimated as

    t_full = t_sample * r,   r = t(polymul, N = 2^16) / t(polymul, N_sample),

with r measured on the same host (ring products dominate the oracle's time).

A query is timed a stage at a time (the client's encryption, each bottom
layer, the lookup, the interaction, each top layer with the decryption after
the last one; dlrm.infer_stages), so that one timed step stays bounded:
`step()` runs the next stage of the current query and starts a new query
after the last.  A query's time is the sum of its stages' times.

Bounded sample (--budget, bench.py's cpu_baseline): the UCI-shaped model's
whole queries (at N = 2^13 one takes seconds), the median of 3; the
Criteo-shaped model's first two stages (the client's encryption and the
first bottom layer, with only that layer's keys), the median of 3, divided
by the share of a query they took when whole queries were timed on the
development host (STAGE_SHARES; 8 x86 cores, one query, N = 2^15).

Usage: python -m oracle.bench_sample --workload criteo --steps 12 --warmup 0
prints one JSON object.  --threads sets OMP_NUM_THREADS for the oracle's C
core (it must be set before the core loads; this module sets it from the
flag before importing it).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

SAMPLE_LOG_N = {"uci": 13, "uci_silu": 13, "criteo": 15}
# The tiny lookup (--workload tiny) runs at its own N = 2^13: run_tiny.
# Each stage's share of a whole query's time, measured on the development host
# (python -m oracle.bench_sample --workload criteo: 149.6 s per query at N =
# 2^15 on 8 cores; --workload uci --steps 21: 7.37 s at N = 2^13).
STAGE_SHARES = {
    "criteo": [0.0018, 0.0965, 0.2515, 0.0802, 0.0650, 0.2248, 0.0506, 0.1645, 0.0603, 0.0048],
    "uci": [0.0074, 0.2195, 0.1916, 0.3856, 0.0714, 0.1085, 0.0161],
}


def _params(log_n: int, levels: int):
    from . import ckks
    return ckks.Params(log_n, [60] + [40] * levels, 3, 60, 3, 40.0)


def polymul_ratio(log_full: int, log_sample: int, limbs: int = 8, reps: int = 3) -> float:
    from . import ckks

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


class StageCycle:
    """The oracle's inference of one query after another, one stage per step."""

    def __init__(self, workload: str, seed: int = 500, key_stages: int = 0):
        """key_stages > 0: rotation keys only for the first key_stages stages
        (the client's encryption, then the bottom layers in order)."""
        from paper_2506_18150_gb300 import synthetic as syn

        from . import ckks, dlrm
        self.ckks, self.dlrm = ckks, dlrm
        spec = {"uci": syn.uci_spec, "criteo": syn.criteo_spec, "uci_silu": syn.uci_silu_spec}[workload](0)
        w = syn.make_weights(spec, 0)
        self.log_n = SAMPLE_LOG_N[workload]
        n_bot, n_top = len(w.bottom_W), len(w.top_W)
        ad = dlrm.activation_levels(spec)
        levels = (1 + ad) * (n_top - 1) + 1 + 2 + (1 + ad) * n_bot     # dot interaction
        self.p = _params(self.log_n, levels)
        t0 = time.perf_counter()
        self.c = dlrm.compile_model(self.p, spec, w)
        steps = self.c.rotation_steps()
        if key_stages:
            from . import linear
            steps = sorted(set().union(*[set(linear.rotation_steps(lay.pm))
                                         for lay in self.c.bottom[:max(0, key_stages - 1)]]))
        self.sk, self.keys = ckks.keygen(self.p, 1, rot_steps=steps)
        self.setup_s = time.perf_counter() - t0
        self.spec, self.seed = spec, seed
        self.q = -1
        self.pending = []
        self.n_stages = 1 + n_bot + 2 + n_top

    def _next_query(self):
        self.q += 1
        dense, idx = self.spec_query(self.q)
        st = {}

        def client():
            st["cd"], st["cs"] = self.dlrm.encrypt_query(self.p, self.keys, self.c, dense, idx,
                                                         self.seed + 2 * self.q)
            stages, st["s"] = self.dlrm.infer_stages(self.p, self.keys, self.c, st["cd"], st["cs"])
            self.pending.extend(stages[:-1])
            self.pending.append(lambda: (stages[-1](), self.dlrm.decrypt_logit(self.p, self.sk, st["s"]["y"])))
        self.pending.append(client)

    def spec_query(self, q: int):
        from paper_2506_18150_gb300 import synthetic as syn
        dense, idx = syn.make_queries(self.spec, 1, seed=self.seed + q)
        return dense[0], idx[0]

    def step(self):
        """Run the next stage; returns (query index, stage index, seconds)."""
        if not self.pending:
            self._next_query()
            self.k = 0
        stage = self.k
        self.k += 1
        f = self.pending.pop(0)
        t0 = time.perf_counter()
        f()
        return self.q, stage, time.perf_counter() - t0


def query_time(records, n_stages: int) -> float:
    """A query's time from stage records: the mean time of each stage index
    over the records, summed over the stages (every stage must appear)."""
    per = [[t for _, s, t in records if s == k] for k in range(n_stages)]
    missing = [k for k, v in enumerate(per) if not v]
    if missing:
        raise ValueError(f"stages {missing} were not timed; run at least {n_stages} steps")
    return float(sum(np.mean(v) for v in per))


def cores() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run(workload: str = "uci", steps: int = 0, warmup: int = 0):
    """Time `warmup` untimed then `steps` timed stages (steps = 0: one whole
    query after the warm-up).  A query's time comes from the timed stages'
    means (STAGE_SHARES fills in stages the run did not time);
    steps_in_queries is the part of a query the timed stages cover."""
    cyc = StageCycle(workload)
    for _ in range(warmup):
        cyc.step()
    n = steps or cyc.n_stages
    t0 = time.perf_counter()
    recs = [cyc.step() for _ in range(n)]
    wall = time.perf_counter() - t0
    r = polymul_ratio(16, cyc.log_n)
    per = [[t for _, s, t in recs if s == k] for k in range(cyc.n_stages)]
    seen = [k for k in range(cyc.n_stages) if per[k]]
    shares = STAGE_SHARES.get(workload)
    if len(seen) == cyc.n_stages:
        tq = query_time(recs, cyc.n_stages)
        how = "every stage timed"
    elif shares:
        tq = sum(float(np.mean(per[k])) for k in seen) / sum(shares[k] for k in seen)
        how = f"stages {seen} timed, the rest from their development-host shares"
    else:
        raise ValueError(f"{n} steps do not cover every stage of {workload}")
    units = sum(t for _, _, t in recs) / tq
    sample = (f"{n} stages of {workload} queries (each stage: the client's encryption, one layer, the lookup or "
              f"the interaction; {cyc.n_stages} per query) at N=2^{cyc.log_n}, {how}; a query = "
              f"{tq:.2f} s there, scaled x{r:.2f} to N=2^16 (the oracle's measured ring-product time ratio)")
    return {"workload": workload, "sample_log_n": cyc.log_n, "n_stages": cyc.n_stages, "steps": n,
            "stage_times_s": [t for _, _, t in recs], "stage_index": [s for _, s, _ in recs],
            "wall_s": wall, "sample_s_per_query": tq, "ratio_to_full": r, "est_full_s_per_query": tq * r,
            "steps_in_queries": units, "setup_s": cyc.setup_s, "cores": cores(), "sample": sample}


def run_tiny(steps: int = 3, exact: bool = False):
    """The tiny lookup (one 1024 x 16 table in base 32 at N = 2^13, three
    50-bit primes and one special prime): per step one query's selector
    (index uniform on 0..1023, seeded), its encoding and encryption, the
    lookup (one BSGS matvec with its folds) and the decryption of the 16
    outputs.  exact: every ring product of the lookup by the schoolbook
    convolution (ckks.EXACT); the keys are made before, the same either way.
    Returns the median time per lookup (no ring-degree scaling: N is the
    workload's own)."""
    from paper_2506_18150_gb300 import synthetic as syn

    from . import ckks, dlrm, linear
    pr = syn.PARAMS["tiny"]
    p = ckks.Params(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"])
    C = syn.tiny_table(0)
    pm = linear.prepare(p, dlrm.lookup_matrix(C, 32, 1024), 64, 16, 1, p.delta, p.delta)
    sk, keys = ckks.keygen(p, 0, rot_steps=linear.rotation_steps(pm))
    times, err = [], 0.0
    for q in range(steps):
        i = int(np.random.default_rng(q).integers(0, 1024))
        t0 = time.perf_counter()
        ckks.EXACT = exact
        try:
            sel = dlrm.replicate(dlrm.selector_vector([1024], 32, [i]), 64, p.n)
            ct = ckks.encrypt(p, keys, ckks.encode_real(p, sel, p.delta), 1, p.delta, 42 + q)
            y = ckks.decrypt(p, sk, linear.matvec(p, keys, pm, ct), 16)
        finally:
            ckks.EXACT = False
        times.append(time.perf_counter() - t0)
        err = max(err, float(np.max(np.abs(y - (C[0][i % 32].astype(np.float64) + C[1][i // 32])))))
    med = float(np.median(times))
    kind = "oracle-exact (schoolbook products)" if exact else "oracle (textbook-NTT products)"
    return {"workload": "tiny", "exact": exact, "times_s": times, "s_per_lookup": med, "max_abs_err": err,
            "cores": cores(), "sample": f"{steps} lookups at N=2^13 (the workload's own size), {kind}, "
                                        f"median {med:.3f} s"}


def run_boot(log_n: int = 12, n_s: int = 512, reps: int = 1):
    """One bootstrap (oracle/boot.py) on the bootstrappable chain (q_0, 13 x
    40-bit, 13 x 60-bit, 3 special primes: the same limbs per operation as at
    N = 2^16) at N = 2^log_n, n_s slots, keys made before the timing.  Each
    stage is timed; SubSum takes log2(N / (2 n_s)) rotations, so its time is
    scaled to the full size's count before the ring-product ratio is applied."""
    from paper_2506_18150_gb300 import synthetic as syn

    from . import boot, ckks
    pr = syn.boot_params(log_n)
    p = ckks.Params(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"])
    t0 = time.perf_counter()
    b = boot.prepare(p, boot.BootParams(n_s=n_s))
    sk, keys = ckks.keygen(p, 7, rot_steps=b.rotation_steps(), h=192, conj=True)
    setup = time.perf_counter() - t0
    z = np.random.default_rng(1).uniform(-1, 1, n_s)[np.arange(p.n) % n_s]
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, z, p.delta), 0, p.delta, 11)
    runs, err = [], 0.0
    for _ in range(reps):
        st = {}
        tt = {}
        x = ct
        t = time.perf_counter()
        x = boot.mod_raise(p, boot.boost(p, x, b.bp.log2_boost))
        tt["raise"] = time.perf_counter() - t
        t = time.perf_counter()
        x = boot.subsum(p, keys, x, b.subsum_steps)
        tt["subsum"] = time.perf_counter() - t
        t = time.perf_counter()
        y = boot.eval_mod(p, keys, b, boot.coeff_to_slot(p, keys, b, x))
        tt["cts_evalmod"] = time.perf_counter() - t
        t = time.perf_counter()
        out = boot.slot_to_coeff(p, keys, b, y, ct.scale)
        tt["stc"] = time.perf_counter() - t
        runs.append(tt)
        err = max(err, float(np.max(np.abs(ckks.decrypt(p, sk, out) - z))))
    full_steps = (1 << 15).bit_length() - 1 - (n_s.bit_length() - 1)      # log2(2^15 / n_s)
    k = full_steps / max(1, len(b.subsum_steps))
    tot = [r["raise"] + k * r["subsum"] + r["cts_evalmod"] + r["stc"] for r in runs]
    med = float(np.median(tot))
    ratio = polymul_ratio(16, log_n)
    return {"workload": "boot", "sample_log_n": log_n, "n_s": n_s, "stage_times_s": runs, "max_abs_err": err,
            "sample_s_per_boot": med, "ratio_to_full": ratio, "est_full_s_per_boot": med * ratio,
            "setup_s": setup, "cores": cores(),
            "sample": (f"{reps} bootstrap(s) of n_s={n_s} slots at N=2^{log_n} on the bootstrappable chain "
                       f"({med:.2f} s, SubSum's {len(b.subsum_steps)} rotations scaled to the {full_steps} of "
                       f"N=2^16), scaled x{ratio:.2f} to N=2^16 (the oracle's measured ring-product time ratio)")}


def run_budget(workload: str, reps: int = 3):
    """The bounded sample of bench.py's cpu_baseline: the median of `reps`
    whole queries (UCI-shaped), or of `reps` runs of the first two stages
    scaled by their share (Criteo-shaped)."""
    first = 2 if workload == "criteo" else 0
    cyc = StageCycle(workload, key_stages=first)
    r = polymul_ratio(16, cyc.log_n)
    runs = []
    for _ in range(reps):
        recs = []
        while True:
            recs.append(cyc.step())
            if (first and len(recs) == first) or (not first and not cyc.pending):
                break
        cyc.pending.clear()
        runs.append(sum(t for _, _, t in recs))
    med = float(np.median(runs))
    if first:
        share = sum(STAGE_SHARES[workload][:first])
        tq = med / share
        sample = (f"the client's encryption and the first bottom layer of a {workload} query at "
                  f"N=2^{cyc.log_n} (median of {reps}: {med:.2f} s), divided by their share of a query "
                  f"({share:.4f}, measured on the development host) and scaled x{r:.2f} to N=2^16 (the "
                  f"oracle's measured ring-product time ratio)")
    else:
        tq = med
        sample = (f"whole {workload} queries at N=2^{cyc.log_n} (median of {reps}: {med:.2f} s), scaled "
                  f"x{r:.2f} to N=2^16 (the oracle's measured ring-product time ratio)")
    return {"workload": workload, "sample_log_n": cyc.log_n, "runs_s": runs, "sample_s_per_query": tq,
            "ratio_to_full": r, "est_full_s_per_query": tq * r, "setup_s": cyc.setup_s, "cores": cores(),
            "sample": sample}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="uci")
    ap.add_argument("--steps", type=int, default=0, help="timed stages (0: one whole query)")
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0, help="OMP_NUM_THREADS for the oracle (0: all cores)")
    ap.add_argument("--budget", action="store_true", help="the bounded sample of bench.py's cpu_baseline")
    ap.add_argument("--exact", action="store_true", help="tiny: schoolbook products (oracle-exact)")
    a = ap.parse_args()
    if a.threads:
        os.environ["OMP_NUM_THREADS"] = str(a.threads)
    if a.workload == "tiny":
        print(json.dumps(run_tiny(a.steps or 3, a.exact)))
    elif a.workload == "boot":
        print(json.dumps(run_boot(reps=a.steps or 1)))
    else:
        print(json.dumps(run_budget(a.workload) if a.budget else run(a.workload, a.steps, a.warmup)))
