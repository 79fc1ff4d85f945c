"""Bit-exact parity of the Criteo-shaped DLRM at the full parameter set
(N = 2^16, q_0 60-bit + 20 x 40-bit, K = 3 x 60-bit special primes,
alpha = 3) against the oracle's results in tests/golden/criteo_n16.json,
which tests/golden/make_criteo_n16.py computes with the oracle alone (about
13 minutes of host time, too long for every run).

Every input is an integer (keys from the ChaCha20 seed, plaintexts from
synthetic.int_poly), so both sides start from the same words on any machine.
Compared word for word (SHA-256 of the coefficient-domain output, with the
first words of each limb to locate a mismatch):

  * one double-hoisted BSGS product (with its rescale and folds) for every
    distinct matrix shape and level of the model -- the kernel instances
    only this model reaches: 6 and 5 digits at levels 15 and 13 (the
    512- and 256-wide bottom layers), D = 512 with 64 baby and 8 giant steps
    at level 8 (the lookup) and level 5 (the 367 -> 512 top layer), the
    256 -> 1 layer with 4 fold levels;
  * one whole inference, through the path the benchmark times (the server
    path of a batch of one captured as a CUDA graph, then replayed) and
    through helrm_infer (every kernel launched on the stream).
"""
import hashlib
import json
import os

import numpy as np
import pytest

from helpers import gpu_ctx

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "criteo_n16.json")))
R = GOLD["recipe"]


def _check(coeffs, level, case):
    assert level == case["level"], (level, case["level"])
    c0, c1 = coeffs[0], coeffs[1]
    for name, poly in (("c0", c0), ("c1", c1)):
        head = np.array(case[f"{name}_head"], dtype=np.uint64)
        bad = [i for i in range(head.shape[0]) if not np.array_equal(poly[i, :4], head[i])]
        assert not bad, f"{name} differs from the oracle in limbs {bad}"
    data = np.concatenate([np.ascontiguousarray(c0, dtype="<u8").reshape(-1),
                           np.ascontiguousarray(c1, dtype="<u8").reshape(-1)])
    assert hashlib.sha256(data.tobytes()).hexdigest() == case["sha256"], "ciphertext differs from the oracle"


@pytest.fixture(scope="module")
def full():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]
    assert R["params"] == pr
    ctx = gpu_ctx(pr)
    spec = syn.criteo_spec(0)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    steps = H.helrm_model_rotations(ctx, model)
    assert steps == R["rotation_steps"]
    sk, evk = H.helrm_keygen(ctx, R["key_seed"], steps)
    return ctx, model, evk, 1 << pr["log_n"], 2.0 ** pr["log2_scale"]


@pytest.mark.parametrize("name", sorted(k for k in GOLD["cases"] if k.startswith("matvec")))
def test_criteo_matvec_full(full, name):
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    ctx, _, evk, n, delta = full
    case = GOLD["cases"][name]
    k, seed, bound = case["index"], R["seed_matvec"] + case["index"], R["bound"]
    pm = H.helrm_ptmat_prepare(ctx, np.ones((case["rows"], case["cols"])), case["in_pad"], case["out_pad"],
                               case["level_in"], delta, delta)
    info = H.helrm_ptmat_info(ctx, pm)
    assert (info["D"], info["n1"], info["n2"], info["nonzero"]) == (case["D"], case["n1"], case["n2"],
                                                                   case["n_diagonals"])
    H.helrm_ptmat_import(ctx, pm, np.stack([syn.int_poly(seed, 1 + j, n, bound)
                                            for j in range(case["n_diagonals"])]))
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, syn.int_poly(seed, 0, n, bound), case["level_in"], delta),
                         300 + k)
    coeffs, lvl, _ = H.helrm_ct_export(ctx, H.helrm_ptct_matvec(ctx, evk, pm, ct))
    _check(coeffs, lvl, case)


def test_criteo_inference_full(full):
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    ctx, model, evk, n, delta = full
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


def test_criteo_products_with_radix4_transforms(monkeypatch):
    """Two of the products again on a context whose transforms all run with
    4 elements per thread (radix-4 rounds, HELRM_NTT_EPT=4), fused base
    conversions and merged rescales included: the same words."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    monkeypatch.setenv("HELRM_NTT_EPT", "4")
    pr = syn.PARAMS["full"]
    ctx = gpu_ctx(pr)
    spec = syn.criteo_spec(0)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    _, evk = H.helrm_keygen(ctx, R["key_seed"], H.helrm_model_rotations(ctx, model))
    for name in ("matvec_13_512x256", "matvec_1_256x1"):
        test_criteo_matvec_full((ctx, model, evk, 1 << pr["log_n"], 2.0 ** pr["log2_scale"]), name)


def test_criteo_batched_and_served_full(full):
    """The lockstep batch path and the serving loop at full size: a batch of
    two queries (the stored query twice, one key set) and a served trace of
    two requests give the stored oracle words for every query."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    ctx, model, evk, n, delta = full
    case = GOLD["cases"]["inference"]
    H.helrm_model_import_plaintexts(ctx, model, np.stack([syn.int_poly(R["seed_model"], k, n, R["bound"])
                                                          for k in range(case["n_plaintexts"])]))
    md, ms = (syn.int_poly(R["seed_query"], j, n, R["bound"]) for j in range(2))
    cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, R["lvl_dense"], delta), 40)
    cs = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, R["lvl_sel"], delta), 41)
    batch = H.helrm_batch_create(ctx, model, [evk, evk])
    for y in H.helrm_infer_batch(ctx, batch, [cd, cd], [cs, cs]):
        coeffs, lvl, _ = H.helrm_ct_export(ctx, y)
        _check(coeffs, lvl, case)
    srv = H.helrm_server_create(ctx, 2, 2, 0)
    H.helrm_server_add_client(ctx, srv, model, evk)
    outs, lat, st = H.helrm_server_run(ctx, srv, [0.0, 0.0, 0.0], [0, 0, 0], [cd, cd, cd], [cs, cs, cs])
    assert st["max_batch"] == 2                      # the first request alone, then a batch of two
    for y in outs:
        coeffs, lvl, _ = H.helrm_ct_export(ctx, y)
        _check(coeffs, lvl, case)
