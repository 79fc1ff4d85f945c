"""Bit-exact parity of the UCI-shaped DLRM with polynomial (SiLU) activations
at the full parameter set, against the oracle's result stored in
tests/golden/uci_silu_n16.json (written by tests/golden/make_criteo_n16.py
--model uci_silu with the oracle alone).

The model's activations are the degree-6 SiLU polynomial with coefficients
rounded to multiples of 2^-20 (synthetic.uci_silu_fixed_spec), its plaintexts
and the query are integers from synthetic.int_poly, and the keys come from
the ChaCha20 seed, so both sides start from the same words on any machine.
Compared word for word: one whole inference through the graph-replayed
batch of one (the polynomial evaluations, their relinearisations and the
constant terms on the layer outputs, at levels 18 down to 0) and through
helrm_infer."""
import hashlib
import json
import os

import numpy as np
import pytest

from helpers import gpu_ctx

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "uci_silu_n16.json")))
R = GOLD["recipe"]


def _check(coeffs, level, case):
    assert level == case["level"], (level, case["level"])
    for name, poly in (("c0", coeffs[0]), ("c1", coeffs[1])):
        head = np.array(case[f"{name}_head"], dtype=np.uint64)
        bad = [i for i in range(head.shape[0]) if not np.array_equal(poly[i, :4], head[i])]
        assert not bad, f"{name} differs from the oracle in limbs {bad}"
    data = np.concatenate([np.ascontiguousarray(coeffs[0], dtype="<u8").reshape(-1),
                           np.ascontiguousarray(coeffs[1], dtype="<u8").reshape(-1)])
    assert hashlib.sha256(data.tobytes()).hexdigest() == case["sha256"], "ciphertext differs from the oracle"


def test_uci_silu_inference_full():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]
    assert R["params"] == pr
    ctx = gpu_ctx(pr)
    n, delta = 1 << pr["log_n"], 2.0 ** pr["log2_scale"]
    spec = syn.uci_silu_fixed_spec(0)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    steps = H.helrm_model_rotations(ctx, model)
    assert steps == R["rotation_steps"]
    _, evk = H.helrm_keygen(ctx, R["key_seed"], steps)
    case = GOLD["cases"]["inference"]
    info = H.helrm_model_info(ctx, model)
    assert info["n_plaintexts"] == case["n_plaintexts"]
    assert (info["lvl_dense"], info["lvl_sel"]) == (R["lvl_dense"], R["lvl_sel"])
    H.helrm_model_import_plaintexts(ctx, model, np.stack([syn.int_poly(R["seed_model"], k, n, R["bound"])
                                                          for k in range(case["n_plaintexts"])]))
    md, ms = (syn.int_poly(R["seed_query"], j, n, R["bound"]) for j in range(2))
    cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, R["lvl_dense"], delta), 40)
    cs = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, R["lvl_sel"], delta), 41)
    batch = H.helrm_batch_create(ctx, model, [evk])
    H.helrm_batch_set_graph(ctx, batch, True)
    for _ in range(2):                                # the capture, then a replay
        coeffs, lvl, _ = H.helrm_ct_export(ctx, H.helrm_infer_batch(ctx, batch, [cd], [cs])[0])
        _check(coeffs, lvl, case)
    coeffs, lvl, _ = H.helrm_ct_export(ctx, H.helrm_infer(ctx, evk, model, cd, cs))
    _check(coeffs, lvl, case)
