"""Kernel micro-benchmarks on caller-owned device buffers.

  python -m paper_2506_18150_gb300.microbench ntt --limbs 192 --reps 20 [--per 20]
  python -m paper_2506_18150_gb300.microbench rotate --level 8 --reps 20

`multi` times the embedding lookup with a selector of --cts ciphertexts.
`ntt` transforms `limbs` limbs of N = 2^16 words (forward then inverse) and
reports the time per limb and the algorithmic bandwidth (16 N bytes per limb
and direction).  `rotate` times one rotation (ModUp, fused automorphism + key
inner product, ModDown) at a level of the full parameter set.  Buffers are a
few hundred MB: larger than L2, small enough for a profiler capture.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def _ctx(torch):
    from . import helrm as H
    from . import synthetic as syn
    pr = syn.PARAMS["full"]
    return H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"],
                              pr["log2_scale"], device=torch.cuda.current_device(),
                              stream=torch.cuda.current_stream().cuda_stream), pr


def bench_ntt(limbs: int, reps: int, per: int = 20):
    import torch

    from . import helrm as H
    ctx, pr = _ctx(torch)
    n = 1 << pr["log_n"]
    primes, _ = H.helrm_ctx_primes(ctx)
    q = primes[1]
    buf = torch.randint(0, q, (limbs * n,), dtype=torch.int64, device="cuda")
    # limbs cycle over the 40-bit primes 1..20 (one launch per block of `per` limbs)
    groups = [(i, min(per, limbs - i)) for i in range(0, limbs, per)]

    def run(inverse):
        for off, cnt in groups:
            H.helrm_ntt(ctx, buf.data_ptr() + off * n * 8, cnt, 1, inverse)

    for _ in range(2):
        run(False)
        run(True)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, inv in [("forward", False), ("inverse", True)]:
        s.record()
        for _ in range(reps):
            run(inv)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / reps
        out[name] = {"ms": ms, "us_per_limb": 1000 * ms / limbs,
                     "GBps_algorithmic": 16.0 * n * limbs / (ms / 1000) / 1e9}
    return out


def bench_rotate(level: int, reps: int):
    import torch

    from . import helrm as H
    ctx, pr = _ctx(torch)
    sk, evk = H.helrm_keygen(ctx, 1, [1])
    z = np.random.default_rng(0).uniform(-1, 1, 1 << (pr["log_n"] - 1))
    ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, z, level, 2.0**40), 3)
    for _ in range(2):
        H.helrm_rotate(ctx, evk, ct, 1)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        H.helrm_rotate(ctx, evk, ct, 1)
    e.record()
    torch.cuda.synchronize()
    return {"level": level, "ms_per_rotation": s.elapsed_time(e) / reps}


def bench_matvec(D: int, level: int, reps: int):
    """One BSGS matvec with a D x D dense matrix at `level` on a chain of
    level+1 ciphertext primes (N = 2^16, same prime sizes as the full set), so
    the rotation keys stay a few GB."""
    import torch

    from . import helrm as H
    ctx = H.helrm_ctx_create(16, [60] + [40] * level, 3, 60, 3, 40.0, device=torch.cuda.current_device(),
                             stream=torch.cuda.current_stream().cuda_stream)
    W = np.random.default_rng(1).normal(0, 0.1, (D, D))
    m = H.helrm_ptmat_prepare(ctx, W, D, D, level, 2.0**40, 2.0**40)
    sk, evk = H.helrm_keygen(ctx, 1, H.helrm_ptmat_rotations(ctx, m))
    x = np.random.default_rng(2).uniform(-1, 1, D)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, np.tile(x, (1 << 15) // D), level, 2.0**40), 3)
    for _ in range(2):
        H.helrm_ptct_matvec(ctx, evk, m, ct)
    torch.cuda.synchronize()
    H.helrm_ctx_profile(ctx, True)
    for _ in range(reps):
        H.helrm_ptct_matvec(ctx, evk, m, ct)
    rep = H.helrm_ctx_profile_report(ctx)
    H.helrm_ctx_profile(ctx, False)
    info = H.helrm_ptmat_info(ctx, m)
    return {"D": D, "level": level, "n1": info["n1"], "n2": info["n2"],
            "kernels": {k: {"ms_per_matvec": v[1] / reps, "GBps": v[2] / (v[1] / 1000) / 1e9 if v[1] else None}
                        for k, v in rep.items()},
            "ms_per_matvec": sum(v[1] for v in rep.values()) / reps}


def bench_multi(n_cts: int, level: int, reps: int):
    """The embedding lookup with a selector of n_cts ciphertexts (HE-LRM Sec.
    5.4: 18 and 85 for the least compressed Criteo models): 26 plain tables
    of n_cts * 2^15 / 26 rows each, 416 outputs (padded to 512), prepared at
    `level` on a chain of level+1 primes (N = 2^16).  Reports ms per lookup."""
    import torch

    from . import helrm as H
    ctx = H.helrm_ctx_create(16, [60] + [40] * level, 3, 60, 3, 40.0, device=torch.cuda.current_device(),
                             stream=torch.cuda.current_stream().cuda_stream)
    n = 1 << 15
    rows = (n_cts * n) // 26
    cards = [rows] * 26
    rng = np.random.default_rng(5)
    tables = [[rng.uniform(-0.05, 0.05, (rows, 16)).astype(np.float32)] for _ in cards]
    emb = H.helrm_emb_prepare(ctx, cards, rows, 0, 16, tables, 0, 512, level, 2.0**40, 2.0**40)
    chunks = H.helrm_emb_chunks(ctx, emb)
    mats = [H.helrm_emb_matrix(ctx, emb, c) for c in range(chunks)]
    steps = sorted(set().union(*[set(H.helrm_ptmat_rotations(ctx, m)) for m in mats]))
    sk, evk = H.helrm_keygen(ctx, 1, steps)
    idx = [int(v) for v in rng.integers(0, rows, 26)]
    slots = H.helrm_query_pack(ctx, emb, idx, chunks * n)
    cts = [H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, slots[c * n:(c + 1) * n], level, 2.0**40), 10 + c)
           for c in range(chunks)]
    y = H.helrm_embedding_lookup_multi(ctx, evk, emb, cts)
    got = H.helrm_decrypt(ctx, sk, y, 416)
    want = np.concatenate([tables[t][0][idx[t]].astype(np.float64) for t in range(26)])
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(reps):
        H.helrm_embedding_lookup_multi(ctx, evk, emb, cts)
    s1.record()
    torch.cuda.synchronize()
    return {"ciphertexts": chunks, "selector_slots": 26 * rows, "outputs": 416, "level": level,
            "ms_per_lookup": s0.elapsed_time(s1) / reps, "max_abs_err": float(np.max(np.abs(got - want)))}


def bench_boot_matvec(log_n: int, n_s: int, reps: int):
    """The CoeffToSlot product of a bootstrap (its BSGS matvec at the top of
    the bootstrappable chain: 9 key-switching digits) on a ciphertext of
    n_s-periodic slots at N = 2^log_n, with keys for its rotations only; the
    first product is a warm-up.  Reports ms per product per kernel family."""
    import torch

    from . import helrm as H
    from . import synthetic as syn
    pr = syn.boot_params(log_n)
    ctx = H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"],
                             device=torch.cuda.current_device(), stream=torch.cuda.current_stream().cuda_stream)
    bt = H.helrm_boot_create(ctx, n_s)
    m = H.helrm_boot_matrix(ctx, bt, 0)
    _, evk = H.helrm_keygen_ex(ctx, 5, 192, H.helrm_ptmat_rotations(ctx, m))
    n = 1 << (log_n - 1)
    z = np.random.default_rng(1).uniform(-1, 1, n_s)
    top = len(pr["q_bits"]) - 1
    ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, z[np.arange(n) % n_s], top, 2.0**40), 4)
    H.helrm_ptct_matvec(ctx, evk, m, ct)
    torch.cuda.synchronize()
    H.helrm_ctx_profile(ctx, True)
    for _ in range(reps):
        H.helrm_ptct_matvec(ctx, evk, m, ct)
    rep = H.helrm_ctx_profile_report(ctx)
    H.helrm_ctx_profile(ctx, False)
    return {"log_n": log_n, "n_s": n_s, "level": top,
            "kernels": {k: {"ms_per_product": v[1] / reps, "GBps": v[2] / (v[1] / 1000) / 1e9 if v[1] else None}
                        for k, v in rep.items()}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["ntt", "rotate", "matvec", "multi", "boot_matvec"])
    ap.add_argument("--log-n", type=int, default=14, help="boot_matvec: ring degree 2^log_n")
    ap.add_argument("--ns", type=int, default=256, help="boot_matvec: slot period")
    ap.add_argument("--cts", type=int, default=18)
    ap.add_argument("--D", type=int, default=256)
    ap.add_argument("--limbs", type=int, default=192)
    ap.add_argument("--level", type=int, default=8)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--per", type=int, default=20, help="ntt: limbs per launch")
    a = ap.parse_args()
    if a.what == "ntt":
        r = bench_ntt(a.limbs, a.reps, a.per)
    elif a.what == "rotate":
        r = bench_rotate(a.level, a.reps)
    elif a.what == "multi":
        r = bench_multi(a.cts, a.level, a.reps)
    elif a.what == "boot_matvec":
        r = bench_boot_matvec(a.log_n, a.ns, a.reps)
    else:
        r = bench_matvec(a.D, a.level, a.reps)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
