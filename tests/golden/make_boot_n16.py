"""Writes tests/golden/boot_n16.json: what the oracle computes for one
bootstrap at the full bootstrappable parameter set (N = 2^16, q_0 60-bit,
13 x 40-bit and 13 x 60-bit primes, 3 x 60-bit special primes, alpha = 3,
a secret with 192 non-zero coefficients), n_s = 512 slots, for the full-size
GPU parity test (tests/test_gpu_boot_full.py).

Only oracle/ and the seeded input generators run here.  Every input is an
integer or a dyadic rational, so the stored results do not depend on the
machine: the keys come from the oracle's ChaCha20 streams (seed 91); the
diagonals of CoeffToSlot and SlotToCoeff are synthetic.int_poly integers
instead of FP64 encodings of the slot matrix (whose last-bit rounding can
differ between machines); the cosine polynomial is the oracle's fit rounded
to multiples of 2^-44 (synthetic.dyadic); the input ciphertext encrypts
int_poly(SEED_IN, 0) (coefficients below 2^36) at level 0 (encryption seed
5).  The arithmetic on them is the bootstrap's, word for word, whatever the
values mean.

Stored per stage (after ModRaise, SubSum, CoeffToSlot, EvalMod, and the
output): the level, the declared scale, the SHA-256 of the ciphertext in the
coefficient domain (c0 limbs then c1 limbs, little-endian uint64) and the
first 4 words of every limb of c0 and c1.

Usage: python tests/golden/make_boot_n16.py   (about 30 minutes on 8 cores)
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

OUT = os.path.join(HERE, "boot_n16.json")
KEY_SEED, H_SECRET = 91, 192
SEED_DIAG, SEED_IN = 1200, 1201
BOUND_DIAG, BOUND_IN = 1 << 30, 1 << 36
N_S = 512


def ct_digest(ct):
    data = np.concatenate([np.ascontiguousarray(ct.c0, dtype="<u8").reshape(-1),
                           np.ascontiguousarray(ct.c1, dtype="<u8").reshape(-1)])
    return {"level": ct.level, "scale": ct.scale, "sha256": hashlib.sha256(data.tobytes()).hexdigest(),
            "c0_head": [[int(x) for x in row[:4]] for row in ct.c0],
            "c1_head": [[int(x) for x in row[:4]] for row in ct.c1]}


def main():
    from helpers import oracle_keys_pool, oracle_params
    from oracle import boot, ckks
    from paper_2506_18150_gb300 import synthetic as syn

    t0 = time.time()
    pr = syn.boot_params()
    p = oracle_params(pr)
    coeffs = syn.dyadic(boot.cos_fit(24, 6, 16), bits=44)
    b = boot.prepare(p, boot.BootParams(n_s=N_S, coeffs=coeffs))
    k = 0
    for pm in b.cts + [b.stc]:
        for key in pm.ordered_keys():
            pm.pts[key] = syn.int_poly(SEED_DIAG, k, p.N, BOUND_DIAG)
            k += 1
    steps = b.rotation_steps()
    _, keys = oracle_keys_pool(pr, KEY_SEED, steps, h=H_SECRET, conj=True)
    print(f"{len(steps)} rotation keys in {time.time() - t0:.0f} s", flush=True)
    ct = ckks.encrypt(p, keys, syn.int_poly(SEED_IN, 0, p.N, BOUND_IN), 0, p.delta, 5)
    st = {}
    t1 = time.time()
    boot.bootstrap(p, keys, b, ct, st)
    print(f"bootstrap in {time.time() - t1:.0f} s", flush=True)
    res = {"recipe": {"params": pr, "key_seed": KEY_SEED, "h": H_SECRET, "n_s": N_S, "seed_diag": SEED_DIAG,
                      "bound_diag": BOUND_DIAG, "seed_in": SEED_IN, "bound_in": BOUND_IN, "enc_seed": 5,
                      "coeffs": list(coeffs), "rotation_steps": steps, "n_diagonals": k,
                      "diagonals": [len(pm.pts) for pm in b.cts + [b.stc]]},
           "stages": {name: ct_digest(st[name]) for name in ["raised", "subsum", "cts", "evalmod", "out"]}}
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
