"""Bit-exact parity of one bootstrap at the full bootstrappable parameter set
(N = 2^16, 13 x 40-bit + 13 x 60-bit primes, 9 key-switching digits at the
top), n_s = 512, against the oracle's results stored in
tests/golden/boot_n16.json (written by tests/golden/make_boot_n16.py with the
oracle alone).

The inputs are integers or dyadic rationals, so both sides start from the
same words on any machine: the keys from the ChaCha20 seed (sparse secret,
h = 192), the diagonals of both matrices int_poly integers (imported), the
cosine polynomial stored in the file, the input an encryption of an int_poly
plaintext at level 0.  Compared word for word after ModRaise, SubSum,
CoeffToSlot, EvalMod and SlotToCoeff."""
import hashlib
import json
import os

import numpy as np
import pytest

from helpers import gpu_ctx

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "boot_n16.json")))
R = GOLD["recipe"]


def _check(ctx, ct, case):
    from paper_2506_18150_gb300 import helrm as H
    coeffs, level, scale = H.helrm_ct_export(ctx, ct)
    assert level == case["level"], (level, case["level"])
    assert scale == case["scale"], (scale, case["scale"])
    for name, poly in (("c0", coeffs[0]), ("c1", coeffs[1])):
        head = np.array(case[f"{name}_head"], dtype=np.uint64)
        bad = [i for i in range(head.shape[0]) if not np.array_equal(poly[i, :4], head[i])]
        assert not bad, f"{name} differs from the oracle in limbs {bad}"
    data = np.concatenate([np.ascontiguousarray(coeffs[0], dtype="<u8").reshape(-1),
                           np.ascontiguousarray(coeffs[1], dtype="<u8").reshape(-1)])
    assert hashlib.sha256(data.tobytes()).hexdigest() == case["sha256"], "ciphertext differs from the oracle"


def test_bootstrap_full_size_bit_exact():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params()
    assert R["params"] == pr
    ctx = gpu_ctx(pr)
    n = 1 << pr["log_n"]
    bt = H.helrm_boot_create(ctx, R["n_s"], coeffs=R["coeffs"])
    assert H.helrm_boot_rotations(ctx, bt) == R["rotation_steps"]
    k = 0
    for w, cnt in enumerate(R["diagonals"]):
        H.helrm_ptmat_import(ctx, H.helrm_boot_matrix(ctx, bt, w),
                             np.stack([syn.int_poly(R["seed_diag"], k + j, n, R["bound_diag"]) for j in range(cnt)]))
        k += cnt
    assert k == R["n_diagonals"]
    _, evk = H.helrm_keygen_ex(ctx, R["key_seed"], R["h"], R["rotation_steps"], conj=True)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, syn.int_poly(R["seed_in"], 0, n, R["bound_in"]), 0,
                                                     2.0 ** pr["log2_scale"]), R["enc_seed"])
    out, st = H.helrm_bootstrap(ctx, evk, bt, ct, stages=True)
    for name, g in zip(["raised", "subsum", "cts", "evalmod", "out"], st):
        _check(ctx, g, GOLD["stages"][name])
    _check(ctx, out, GOLD["stages"]["out"])
