"""Bit-exact parity of the Criteo-shaped model with SiLU activations and two
bootstraps (before bottom layer 2 and on z) at the full bootstrappable
parameter set (N = 2^16, 13 compute and 13 bootstrapping primes, 9 digits at
the top), against the oracle's result stored in
tests/golden/criteo_silu_boot_n16.json (written by
tests/golden/make_criteo_n16.py --model criteo_silu_boot with the oracle
alone).

Every input is an integer or a dyadic rational: the keys from the ChaCha20
seed (a sparse secret, h = 192), the model's and the bootstraps' plaintexts
int_poly integers in the canonical order, the SiLU coefficients rounded to
2^-20 and the cosine polynomial to 2^-44 (stored in the file), the query two
encryptions of int_poly plaintexts.  Compared word for word: the logit
ciphertext of helrm_infer (bottom MLP, bootstrap, lookup, bootstrap,
interaction, top MLP)."""
import hashlib
import json
import os

import numpy as np
import pytest

from helpers import gpu_ctx

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                   "criteo_silu_boot_n16.json")))
R = GOLD["recipe"]


def test_criteo_silu_with_bootstraps_full_bit_exact():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params()
    assert R["params"] == pr
    ctx = gpu_ctx(pr)
    n, delta = 1 << pr["log_n"], 2.0 ** pr["log2_scale"]
    spec = syn.criteo_silu_boot_fixed_spec(0)
    assert list(spec.act) == R["act"]
    spec.boot_coeffs = tuple(R["boot_coeffs"])
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    assert H.helrm_model_rotations(ctx, model) == R["rotation_steps"]
    case = GOLD["cases"]["inference"]
    info = H.helrm_model_info(ctx, model)
    assert info["n_plaintexts"] == case["n_plaintexts"]
    assert (info["lvl_dense"], info["lvl_sel"]) == (R["lvl_dense"], R["lvl_sel"])
    H.helrm_model_import_plaintexts(ctx, model, np.stack([syn.int_poly(R["seed_model"], k, n, R["bound"])
                                                          for k in range(case["n_plaintexts"])]))
    _, evk = H.helrm_model_keygen(ctx, model, R["key_seed"])
    md, ms = (syn.int_poly(R["seed_query"], j, n, R["bound"]) for j in range(2))
    cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, R["lvl_dense"], delta), 40)
    cs = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, R["lvl_sel"], delta), 41)
    coeffs, lvl, _ = H.helrm_ct_export(ctx, H.helrm_infer(ctx, evk, model, cd, cs))
    assert lvl == case["level"]
    for name, poly in (("c0", coeffs[0]), ("c1", coeffs[1])):
        head = np.array(case[f"{name}_head"], dtype=np.uint64)
        bad = [i for i in range(head.shape[0]) if not np.array_equal(poly[i, :4], head[i])]
        assert not bad, f"{name} differs from the oracle in limbs {bad}"
    data = np.concatenate([np.ascontiguousarray(coeffs[0], dtype="<u8").reshape(-1),
                           np.ascontiguousarray(coeffs[1], dtype="<u8").reshape(-1)])
    assert hashlib.sha256(data.tobytes()).hexdigest() == case["sha256"], "ciphertext differs from the oracle"
