"""Polynomial activations on the GPU (the paper's Criteo models use polynomial
ReLU / SiLU activations, Sec. 2.1.4, Sec. 5.4): helrm_poly_eval bit-exact
against the oracle's evaluation on the same keys and ciphertexts; a DLRM with
the SiLU polynomial bit-exact against the oracle with its plaintexts and
within 1e-3 of the FP64 model; the UCI-shaped SiLU model at the full
parameter set (N = 2^16, ct_dense at level 18)."""
import numpy as np
import pytest

from helpers import assert_ct_equal, gpu_ctx, oracle_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("coeffs", [(0.25, -1.0, 0.0, 2.0), (0.0, 0.5, 0.2, 0.0, -0.01, 0.0, 0.001), (0.0, 1.0)])
def test_poly_eval_bit_exact_against_oracle(coeffs):
    from oracle import ckks, poly
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 6)
    p = oracle_params(pr)
    ctx = gpu_ctx(pr)
    sk, evk = H.helrm_keygen(ctx, 41, [])
    _, keys_o = ckks.keygen(p, 41, rot_steps=[], relin=True)
    x = np.random.default_rng(3).uniform(-1, 1, p.n)
    m = ckks.encode_real(p, x, p.delta)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, 6, p.delta), 91)
    ct_o = ckks.encrypt(p, keys_o, m, 6, p.delta, 91)
    y = H.helrm_poly_eval(ctx, evk, ct, coeffs, p.delta)
    y_o = poly.poly_eval(p, keys_o, ct_o, coeffs, p.delta)
    assert_ct_equal(ctx, y, y_o)
    got = H.helrm_decrypt(ctx, sk, y, 64)
    assert np.max(np.abs(got - np.polynomial.polynomial.polyval(x[:64], np.asarray(coeffs)))) < 1e-4


def test_poly_eval_errors():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 6)
    ctx = gpu_ctx(pr)
    _, evk = H.helrm_keygen(ctx, 42, [])
    ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, np.zeros(8), 2, 2.0**40), 1)
    for coeffs, name in [((1.0, 0.0, 0.0, 0.0, 1.0), "HELRM_E_LEVEL"),   # depth 3 at level 2
                         ((1.0,), "HELRM_E_INVAL"), ((0.0, 1.0, 0.0), "HELRM_E_INVAL")]:
        with pytest.raises(H.HelrmError) as e:
            H.helrm_poly_eval(ctx, evk, ct, coeffs, 2.0**40)
        assert e.value.name == name


def _tiny_silu_spec():
    from paper_2506_18150_gb300 import synthetic as syn
    spec = syn.DLRMSpec("tiny_silu", 4, [4, 16], [0, 1], [3, 5], 8, 16, "dot", act=syn.silu_poly(7))
    spec.top[0] = syn.top_input_width(spec)
    return spec


def test_silu_dlrm_bit_exact_and_accurate():
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(10, 8)
    p = oracle_params(pr)
    spec = _tiny_silu_spec()
    w = syn.make_weights(spec, 0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    c = dlrm.compile_model(p, spec, w)
    info = H.helrm_model_info(ctx, model)
    assert (info["lvl_dense"], info["lvl_sel"], info["lvl_z"], info["lvl_u"]) == (c.lvl_dense, c.lvl_sel, c.lvl_z, c.lvl_u)
    assert info["n_plaintexts"] == len(c.plaintexts())
    steps = H.helrm_model_rotations(ctx, model)
    assert steps == c.rotation_steps()
    sk, evk = H.helrm_keygen(ctx, 5, steps)
    dense, idx = syn.make_queries(spec, 2, seed=8)
    lg, _ = H.helrm_infer_e2e(ctx, sk, evk, model, dense, idx, 11)      # the library's own encoder
    for q in range(2):
        assert abs(lg[q] - dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]) < 1e-3
    # the oracle's plaintexts and the same seeds: the logit ciphertext bit for bit
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    _, keys_o = ckks.keygen(p, 5, rot_steps=c.rotation_steps())
    xd, xs = dlrm.query_slots(p, c, dense[1], idx[1])
    md, ms = ckks.encode_real(p, xd, p.delta), ckks.encode_real(p, xs, p.delta)
    cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 20)
    cs = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, c.lvl_sel, p.delta), 21)
    out_o = dlrm.infer(p, keys_o, c, ckks.encrypt(p, keys_o, md, c.lvl_dense, p.delta, 20),
                       ckks.encrypt(p, keys_o, ms, c.lvl_sel, p.delta, 21))
    assert_ct_equal(ctx, H.helrm_infer(ctx, evk, model, cd, cs), out_o)


def test_uci_silu_full_parameters():
    """UCI-shaped DLRM with the degree-6 SiLU polynomial at N = 2^16, 20
    levels: three activations of depth 4, ct_dense at level 18; decrypted
    logits against the FP64 model with the same polynomial, and the lockstep
    batch gives the one-query logits."""
    from oracle import dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    spec = syn.uci_silu_spec()
    w = syn.make_weights(spec, 0)
    ctx = gpu_ctx(syn.PARAMS["full"])
    model = H.helrm_model_create(ctx, spec, w)
    assert H.helrm_model_info(ctx, model)["lvl_dense"] == 18
    sk, evk = H.helrm_model_keygen(ctx, model, 7)
    dense, idx = syn.make_queries(spec, 3, seed=12)
    lg, _ = H.helrm_infer_e2e(ctx, sk, evk, model, dense, idx, 30)
    for q in range(3):
        ref = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]
        assert abs(lg[q] - ref) < 1e-3, (q, lg[q], ref)
    cts = [H.helrm_encrypt_query(ctx, evk, model, dense[q], idx[q], 30 + 2 * q) for q in range(3)]
    batch = H.helrm_batch_create(ctx, model, [evk] * 3)
    ys = H.helrm_infer_batch(ctx, batch, [a for a, _ in cts], [b for _, b in cts])
    assert [H.helrm_decrypt_logit(ctx, sk, y)[0] for y in ys] == list(lg)
