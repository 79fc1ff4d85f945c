"""GPU parity of the encrypted DLRM: the compiled model (levels, layouts,
plaintext list) matches the oracle's; with the oracle's integer plaintexts the
encrypted logit is bit-exact; with the library's own encoder the decrypted
logit is within 1e-3 of the FP64 cleartext DLRM, at the reduced ring (N=2^13)
and at the full UCI-shaped configuration (N=2^16, 20 levels)."""
import numpy as np
import pytest

from helpers import assert_ct_equal, gpu_ctx, oracle_keys_pool, oracle_params

pytestmark = pytest.mark.gpu


def _setup(interaction, pr, with_oracle=True):
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    spec = syn.uci_spec(0, interaction)
    w = syn.make_weights(spec, 0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    steps = H.helrm_model_rotations(ctx, model)
    sk, evk = H.helrm_keygen(ctx, 1, steps)
    out = dict(spec=spec, w=w, ctx=ctx, model=model, steps=steps, sk=sk, evk=evk)
    if with_oracle:
        p = oracle_params(pr)
        c = dlrm.compile_model(p, spec, w)
        out.update(p=p, comp=c)
    return out


@pytest.fixture(scope="module", params=["dot", "concat"])
def reduced(request):
    from oracle import ckks
    from paper_2506_18150_gb300 import synthetic as syn
    e = _setup(request.param, syn.reduced_params(13, 9))
    e["sk_o"], e["keys_o"] = ckks.keygen(e["p"], 1, rot_steps=e["comp"].rotation_steps())
    return e


def test_model_layout_matches_oracle(reduced):
    from paper_2506_18150_gb300 import helrm as H
    e = reduced
    c = e["comp"]
    info = H.helrm_model_info(e["ctx"], e["model"])
    assert (info["lvl_dense"], info["lvl_sel"], info["lvl_z"], info["lvl_u"]) == (c.lvl_dense, c.lvl_sel, c.lvl_z, c.lvl_u)
    assert (info["p_dense"], info["p_sel"], info["W_z"], info["W_u"]) == (c.p_dense, c.p_sel, c.W_z, c.W_u)
    assert info["n_plaintexts"] == len(c.plaintexts())
    assert e["steps"] == c.rotation_steps()


def test_model_encoder_within_one_unit(reduced):
    from paper_2506_18150_gb300 import helrm as H
    e = reduced
    got = H.helrm_model_export_plaintexts(e["ctx"], e["model"])
    want = np.stack([np.asarray(x, dtype=np.int64) for x in e["comp"].plaintexts()])
    d = np.abs(got - want)
    assert d.max() <= 1
    assert d.sum() <= got.size // 500 + 8


def test_encrypted_logit_bit_exact(reduced):
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    e = reduced
    p, c, ctx = e["p"], e["comp"], e["ctx"]
    H.helrm_model_import_plaintexts(ctx, e["model"],
                                    np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    dense, idx = syn.make_queries(e["spec"], 1, seed=5)
    xd, xs = dlrm.query_slots(p, c, dense[0], idx[0])
    md, ms = ckks.encode_real(p, xd, p.delta), ckks.encode_real(p, xs, p.delta)
    cd = H.helrm_encrypt(ctx, e["evk"], H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 100)
    cs = H.helrm_encrypt(ctx, e["evk"], H.helrm_pt_import(ctx, ms, c.lvl_sel, p.delta), 101)
    out = H.helrm_infer(ctx, e["evk"], e["model"], cd, cs)
    cd_o = ckks.encrypt(p, e["keys_o"], md, c.lvl_dense, p.delta, 100)
    cs_o = ckks.encrypt(p, e["keys_o"], ms, c.lvl_sel, p.delta, 101)
    out_o = dlrm.infer(p, e["keys_o"], c, cd_o, cs_o)
    assert_ct_equal(ctx, out, out_o)
    ref = dlrm.dlrm_cleartext(e["spec"], e["w"], dense[0], idx[0])[0]
    lg, _ = H.helrm_decrypt_logit(ctx, e["sk"], out)
    assert abs(lg - ref) < 1e-3


def _check_e2e(e, n_q, seed):
    from oracle import dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    dense, idx = syn.make_queries(e["spec"], n_q, seed=seed)
    lg, pr = H.helrm_infer_e2e(e["ctx"], e["sk"], e["evk"], e["model"], dense, idx, 7)
    for q in range(n_q):
        ref, ref_p, _ = dlrm.dlrm_cleartext(e["spec"], e["w"], dense[q], idx[q])
        assert abs(lg[q] - ref) < 1e-3 and abs(pr[q] - ref_p) < 1e-3, (q, lg[q], ref)
    # the same queries through the step-by-step API give the same logits
    cd, cs = H.helrm_encrypt_query(e["ctx"], e["evk"], e["model"], dense[0], idx[0], 7)
    lg0, _ = H.helrm_decrypt_logit(e["ctx"], e["sk"], H.helrm_infer(e["ctx"], e["evk"], e["model"], cd, cs))
    assert lg0 == lg[0]


def test_e2e_with_library_encoder_reduced():
    from paper_2506_18150_gb300 import synthetic as syn
    _check_e2e(_setup("dot", syn.reduced_params(13, 9), with_oracle=False), 3, 21)


def test_full_uci_configuration():
    """UCI-shaped DLRM at the full parameter set (N = 2^16, q_0 + 20 x 40-bit,
    three 60-bit special primes): decrypted logits vs the cleartext DLRM."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    e = _setup("dot", syn.PARAMS["full"], with_oracle=False)
    info = H.helrm_model_info(e["ctx"], e["model"])
    assert (info["lvl_dense"], info["lvl_sel"]) == (9, 6)
    _check_e2e(e, 4, 33)


def test_full_criteo_configuration():
    """Criteo-shaped DLRM at the full parameter set: 13 log-normal dense
    features, 26 tables (33.8M rows, base 64, Zipf indices), bottom
    13-512-256-64-16, dot interaction (27 blocks), top 367-512-256-1."""
    from oracle import dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    spec = syn.criteo_spec(0)
    w = syn.make_weights(spec, 0)
    ctx = gpu_ctx(syn.PARAMS["full"])
    model = H.helrm_model_create(ctx, spec, w)
    info = H.helrm_model_info(ctx, model)
    assert (info["lvl_dense"], info["lvl_sel"], info["p_sel"], info["W_u"]) == (15, 8, 8192, 16384)
    sk, evk = H.helrm_keygen(ctx, 3, H.helrm_model_rotations(ctx, model))
    dense, idx = syn.make_queries(spec, 2, seed=9)
    lg, pr = H.helrm_infer_e2e(ctx, sk, evk, model, dense, idx, 11)
    for q in range(2):
        ref, ref_p, _ = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])
        assert abs(lg[q] - ref) < 1e-3 and abs(pr[q] - ref_p) < 1e-3, (q, lg[q], ref)


def test_wrong_query_level_is_rejected():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    e = _setup("concat", syn.reduced_params(13, 9), with_oracle=False)
    dense, idx = syn.make_queries(e["spec"], 1, seed=1)
    cd, cs = H.helrm_encrypt_query(e["ctx"], e["evk"], e["model"], dense[0], idx[0], 3)
    with pytest.raises(H.HelrmError) as ex:
        H.helrm_infer(e["ctx"], e["evk"], e["model"], cs, cd)
    assert ex.value.name == "HELRM_E_LEVEL"
    bad = idx[0].copy()
    bad[0] = e["spec"].cards[0]
    with pytest.raises(H.HelrmError) as ex:
        H.helrm_encrypt_query(e["ctx"], e["evk"], e["model"], dense[0], bad, 3)
    assert ex.value.name == "HELRM_E_INVAL"


def test_criteo_shaped_logit_bit_exact():
    """The Criteo model's structure at a smaller size: 13 dense features, 26
    tables (2..399 rows, base 64), bottom 13-64-16, dot interaction of 27
    blocks (367 = 16 + C(27, 2) top inputs, padded to 512), top 367-64-1.  The
    interaction's layout needs 13 x 1024 slots, so N = 2^15.  With the
    oracle's plaintexts, keys and encryption randomness the logit ciphertext
    is bit-exact; the logit is the FP64 model's within 1e-3."""
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    rng = np.random.default_rng(5)
    spec = syn.DLRMSpec("criteo_small", 13, [13, 64, 16], [0, 64, 1], [int(x) for x in rng.integers(2, 400, 26)],
                        64, 16, "dot")
    spec.top[0] = syn.top_input_width(spec)
    assert spec.top[0] == 367
    pr = syn.reduced_params(15, 9)
    p = oracle_params(pr)
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    steps = c.rotation_steps()
    _, keys_o = oracle_keys_pool(pr, 3, steps)          # the pool starts before this test's first GPU call
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    info = H.helrm_model_info(ctx, model)
    assert (info["lvl_dense"], info["lvl_sel"], info["lvl_z"], info["lvl_u"]) == (c.lvl_dense, c.lvl_sel, c.lvl_z, c.lvl_u)
    assert H.helrm_model_rotations(ctx, model) == steps
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    sk, evk = H.helrm_keygen(ctx, 3, steps)
    dense, idx = syn.make_queries(spec, 1, seed=4)
    xd, xs = dlrm.query_slots(p, c, dense[0], idx[0])
    md, ms = ckks.encode_real(p, xd, p.delta), ckks.encode_real(p, xs, p.delta)
    cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 20)
    cs = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, c.lvl_sel, p.delta), 21)
    y = H.helrm_infer(ctx, evk, model, cd, cs)
    y_o = dlrm.infer(p, keys_o, c, ckks.encrypt(p, keys_o, md, c.lvl_dense, p.delta, 20),
                     ckks.encrypt(p, keys_o, ms, c.lvl_sel, p.delta, 21))
    assert_ct_equal(ctx, y, y_o)
    assert abs(H.helrm_decrypt_logit(ctx, sk, y)[0] - dlrm.dlrm_cleartext(spec, w, dense[0], idx[0])[0]) < 1e-3
