"""Writes tests/golden/criteo_n16.json: what the oracle computes for the
Criteo-shaped DLRM at the full parameter set (N = 2^16, q_0 60-bit + 20 x
40-bit, K = 3 x 60-bit special primes, alpha = 3), for the full-size GPU
parity tests (tests/test_gpu_criteo_full.py).  With --model uci_silu it
writes tests/golden/uci_silu_n16.json, the inference case alone, for the
UCI-shaped model whose activations are the degree-6 SiLU polynomial (its
coefficients rounded to multiples of 2^-20, synthetic.uci_silu_fixed_spec, so
that the model does not depend on the machine's least-squares fit).

Only oracle/ and the seeded input generators run here.  Every input is an
integer, so the stored results do not depend on the machine: the keys come
from the oracle's ChaCha20 streams (seed 77), and every plaintext (the
model's diagonals, biases, masks and ones block; the two query plaintexts;
the matvec inputs and diagonals) is synthetic.int_poly (SplitMix64 counters)
instead of an FP64 encoding, whose last-bit rounding can differ between
machines.  The arithmetic on them is the method's, word for word, whatever
the values mean.

Stored per case: the output level, the SHA-256 of the output ciphertext in
the coefficient domain (c0 limbs then c1 limbs, little-endian uint64), and
the first 4 words of every limb of c0 and c1.

Cases:
  matvec_<level>_<in_pad>x<out_pad>: one double-hoisted BSGS product (with
      its rescale and folds) for every distinct matrix shape and level of
      the model: a fresh ciphertext of int_poly(SEED_MV + k, 0) at the
      level (encryption seed 300 + k), diagonals int_poly(SEED_MV + k, 1 + j)
      in (g, b) order, the structure of a dense matrix of ones of the
      layer's (rows, cols);
  inference: the whole model (bottom MLP, lookup, dot interaction, top MLP)
      with the model's plaintexts int_poly(SEED_MODEL, k) in its canonical
      order, on ct_dense = Enc(int_poly(SEED_QUERY, 0)) at lvl_dense (seed
      40) and ct_sel = Enc(int_poly(SEED_QUERY, 1)) at lvl_sel (seed 41).

With --model criteo_silu_boot it writes tests/golden/criteo_silu_boot_n16.json,
the inference case alone, for the Criteo-shaped model with SiLU activations
and two bootstraps on the bootstrappable chain (synthetic.boot_params(): 13
compute and 13 bootstrapping primes, a secret with 192 non-zero
coefficients): the SiLU and cosine coefficients rounded to multiples of 2^-20
and 2^-44, and the bootstraps' diagonals int_poly integers like every other
plaintext (they follow the model's in the canonical order).

Usage: python tests/golden/make_criteo_n16.py [--model uci_silu | criteo_silu_boot]
(about 13 minutes on 8 cores for the Criteo-shaped model)
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

OUT = os.path.join(HERE, "{model}_n16.json")
KEY_SEED = 77
SEED_MODEL, SEED_QUERY, SEED_MV = 901, 902, 1000
BOUND = 1 << 20


def ct_digest(c0: np.ndarray, c1: np.ndarray):
    data = np.concatenate([np.ascontiguousarray(c0, dtype="<u8").reshape(-1),
                           np.ascontiguousarray(c1, dtype="<u8").reshape(-1)])
    return {"sha256": hashlib.sha256(data.tobytes()).hexdigest(),
            "c0_head": [[int(x) for x in row[:4]] for row in c0],
            "c1_head": [[int(x) for x in row[:4]] for row in c1]}


def matvec_shapes(c):
    """(name, level, rows, cols, in_pad, out_pad) of every distinct product of the compiled model."""
    seen, out = set(), []
    mats = [lay.pm for lay in c.bottom] + c.emb_pms() + [lay.pm for lay in c.top]
    for pm in mats:
        lay = pm.layout
        key = (pm.level, lay.in_pad, lay.out_pad)
        if key in seen:
            continue
        seen.add(key)
        out.append((f"matvec_{pm.level}_{lay.in_pad}x{lay.out_pad}", pm.level, lay.out_pad, lay.in_pad,
                    lay.in_pad, lay.out_pad))
    return out


def main(model: str = "criteo"):
    from helpers import oracle_keys_pool, oracle_params
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import synthetic as syn

    t0 = time.time()
    boots = model == "criteo_silu_boot"
    pr = syn.boot_params() if boots else syn.PARAMS["full"]
    p = oracle_params(pr)
    spec = {"criteo": syn.criteo_spec, "uci_silu": syn.uci_silu_fixed_spec,
            "criteo_silu_boot": syn.criteo_silu_boot_fixed_spec}[model](0)
    if boots:   # the cosine polynomial of the bootstraps: the oracle's fit, rounded to multiples of 2^-44
        from oracle import boot
        spec.boot_coeffs = syn.dyadic(boot.cos_fit(24, 6, 16), bits=44)
    c = dlrm.compile_model(p, spec, syn.make_weights(spec, 0))
    steps = c.rotation_steps()
    _, keys = oracle_keys_pool(pr, KEY_SEED, steps, h=192 if boots else 0, conj=boots)
    print(f"{len(steps)} rotation keys in {time.time() - t0:.0f} s", flush=True)
    res = {"recipe": {"params": pr, "key_seed": KEY_SEED, "seed_model": SEED_MODEL, "seed_query": SEED_QUERY,
                      "seed_matvec": SEED_MV, "bound": BOUND, "rotation_steps": steps,
                      "lvl_dense": c.lvl_dense, "lvl_sel": c.lvl_sel},
           "cases": {}}
    if boots:
        res["recipe"]["boot_coeffs"] = list(spec.boot_coeffs)
        res["recipe"]["act"] = list(spec.act)

    for k, (name, level, rows, cols, ip, op) in enumerate(matvec_shapes(c) if model == "criteo" else []):
        t1 = time.time()
        pm = linear.prepare(p, np.ones((rows, cols)), ip, op, level, p.delta, p.delta)
        for j, key in enumerate(pm.ordered_keys()):
            pm.pts[key] = syn.int_poly(SEED_MV + k, 1 + j, p.N, BOUND)
        ct = ckks.encrypt(p, keys, syn.int_poly(SEED_MV + k, 0, p.N, BOUND), level, p.delta, 300 + k)
        y = linear.matvec(p, keys, pm, ct)
        d = ct_digest(y.c0, y.c1)
        d.update({"index": k, "level_in": level, "rows": rows, "cols": cols, "in_pad": ip, "out_pad": op,
                  "level": y.level, "n_diagonals": len(pm.pts),
                  "D": pm.layout.D, "n1": pm.layout.n1, "n2": pm.layout.n2, "dnum": p.dnum(level)})
        res["cases"][name] = d
        print(f"{name}: D={pm.layout.D} n1={pm.layout.n1} n2={pm.layout.n2} in {time.time() - t1:.0f} s",
              flush=True)

    t1 = time.time()
    pts = c.plaintexts()
    ints = [syn.int_poly(SEED_MODEL, k, p.N, BOUND) for k in range(len(pts))]
    it = iter(ints)
    # the same canonical order as Compiled.plaintexts()
    for lay in c.bottom:
        for key in lay.pm.ordered_keys():
            lay.pm.pts[key] = next(it)
        lay.bias = next(it)
        if lay.act_const is not None:
            lay.act_const = next(it)
    for pm in c.emb_pms():
        for key in pm.ordered_keys():
            pm.pts[key] = next(it)
    if spec.interaction == "dot":
        c.ones = next(it)
        c.masks = [next(it) for _ in c.masks]
    for lay in c.top:
        for key in lay.pm.ordered_keys():
            lay.pm.pts[key] = next(it)
        lay.bias = next(it)
        if lay.act_const is not None:
            lay.act_const = next(it)
    for name in dlrm.boot_order(c):
        bt = c.boots[name][0]
        for pm in bt.cts + [bt.stc]:
            for key in pm.ordered_keys():
                pm.pts[key] = next(it)
    assert next(it, None) is None
    assert all(np.array_equal(a, b) for a, b in zip(c.plaintexts(), ints))
    cd = ckks.encrypt(p, keys, syn.int_poly(SEED_QUERY, 0, p.N, BOUND), c.lvl_dense, p.delta, 40)
    cs = ckks.encrypt(p, keys, syn.int_poly(SEED_QUERY, 1, p.N, BOUND), c.lvl_sel, p.delta, 41)
    y = dlrm.infer(p, keys, c, cd, cs)
    d = ct_digest(y.c0, y.c1)
    d.update({"level": y.level, "n_plaintexts": len(pts)})
    res["cases"]["inference"] = d
    print(f"inference in {time.time() - t1:.0f} s", flush=True)
    out = OUT.format(model=model)
    with open(out, "w") as f:
        json.dump(res, f, indent=1)
    print(f"wrote {out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--model", default="criteo", choices=["criteo", "uci_silu", "criteo_silu_boot"])
    main(ap.parse_args().model)
