"""Selectors wider than the slot count (HE-LRM Sec. 5.4: the least compressed
Criteo models need 18 and 85 input ciphertexts): the selector is split over
ceil(width / n) ciphertexts, each with its own lookup matrix, and the lookup
is the sum of the per-ciphertext BSGS products.  Bit-exact against the
oracle's lookup_multi with its integer plaintexts, and within 1e-3 of the
gathered rows with the library's own encoder."""
import numpy as np
import pytest

from helpers import assert_ct_equal, gpu_ctx, oracle_params

pytestmark = pytest.mark.gpu


def test_two_ciphertext_lookup_bit_exact_and_accurate():
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 3)                    # n = 2048 slots
    p = oracle_params(pr)
    cards, base = [3000, 40], 4096                   # plain one-hots: 3040 selector slots, 2 ciphertexts
    rng = np.random.default_rng(31)
    tables = [[rng.uniform(-0.05, 0.05, (k, 16)).astype(np.float32)] for k in cards]
    ctx = gpu_ctx(pr)
    emb = H.helrm_emb_prepare(ctx, cards, base, 0, 16, tables, 0, 32, 2, p.delta, p.delta)
    assert H.helrm_emb_chunks(ctx, emb) == 2
    M = dlrm.embedding_matrix(cards, base, tables, 0, 32)
    pms = dlrm.prepare_multi(p, M, 32, 2, p.delta, p.delta)
    mats = [H.helrm_emb_matrix(ctx, emb, c) for c in range(2)]
    assert [H.helrm_ptmat_info(ctx, m)["D"] for m in mats] == [pm.layout.D for pm in pms]
    steps = sorted(set().union(*[set(H.helrm_ptmat_rotations(ctx, m)) for m in mats]))
    assert steps == sorted(set().union(*[linear.rotation_steps(pm) for pm in pms]))
    sk, evk = H.helrm_keygen(ctx, 17, steps)
    _, keys_o = ckks.keygen(p, 17, rot_steps=steps, relin=False)
    for idx in [(2999, 0), (5, 39)]:
        sel = dlrm.selector_vector(cards, base, idx)
        x = dlrm.chunk_slots(sel, p.n)
        assert np.array_equal(H.helrm_query_pack(ctx, emb, list(idx), 2 * p.n), np.concatenate(x))
        want = np.concatenate(dlrm.embedding_cleartext(cards, base, tables, idx))
        # library encoder: decrypted lookup vs the gathered rows
        cts = [H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, xi, 2, p.delta), 60 + c) for c, xi in enumerate(x)]
        got = H.helrm_decrypt(ctx, sk, H.helrm_embedding_lookup_multi(ctx, evk, emb, cts), 32)
        assert np.max(np.abs(got - want)) < 1e-3, idx
    # bit-exact with the oracle's integer plaintexts (diagonals and selectors)
    for c in range(2):
        H.helrm_ptmat_import(ctx, mats[c], np.stack([pms[c].pts[k] for k in pms[c].ordered_keys()]).astype(np.int64))
    sel = dlrm.selector_vector(cards, base, (1234, 7))
    ms = [ckks.encode_real(p, xi, p.delta) for xi in dlrm.chunk_slots(sel, p.n)]
    cts = [H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, 2, p.delta), 90 + c) for c, m in enumerate(ms)]
    cts_o = [ckks.encrypt(p, keys_o, m, 2, p.delta, 90 + c) for c, m in enumerate(ms)]
    assert_ct_equal(ctx, H.helrm_embedding_lookup_multi(ctx, evk, emb, cts), dlrm.lookup_multi(p, keys_o, pms, cts_o))
    with pytest.raises(H.HelrmError) as e:      # one ciphertext is not the whole selector
        H.helrm_embedding_lookup(ctx, evk, emb, cts[0])
    assert e.value.name == "HELRM_E_INVAL"


def test_wide_dlrm_with_two_selector_ciphertexts():
    """The wide DLRM (tables of 700, 2000 and 3 rows, base 4, threshold 1000:
    a 727-slot selector) at N = 2^10 (512 slots): the query carries two
    selector ciphertexts and the lookup is the sum of their two BSGS products.
    The compiled model matches the oracle's; with the oracle's plaintexts and
    the same seeds the logit ciphertext is bit-exact; with the library's own
    encoder the logits are within 1e-3 of the FP64 cleartext DLRM; the
    lockstep batch gives the one-query ciphertexts bit for bit."""
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(10, 5)
    p = oracle_params(pr)
    spec = syn.wide_spec()
    w = syn.make_weights(spec, 0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    c = dlrm.compile_model(p, spec, w)
    info = H.helrm_model_info(ctx, model)
    assert info["n_sel"] == c.n_sel() == 2
    assert (info["lvl_dense"], info["lvl_sel"], info["lvl_z"], info["lvl_u"]) == (c.lvl_dense, c.lvl_sel, c.lvl_z, c.lvl_u)
    assert (info["p_dense"], info["p_sel"], info["W_z"], info["W_u"]) == (c.p_dense, c.p_sel, c.W_z, c.W_u)
    assert info["n_plaintexts"] == len(c.plaintexts())
    steps = H.helrm_model_rotations(ctx, model)
    assert steps == c.rotation_steps()
    sk, evk = H.helrm_keygen(ctx, 1, steps)

    # library encoder: the whole protocol, then the step-by-step calls
    dense, idx = syn.make_queries(spec, 3, seed=6)
    lg, prob = H.helrm_infer_e2e(ctx, sk, evk, model, dense, idx, 7)
    for q in range(3):
        ref, ref_p, _ = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])
        assert abs(lg[q] - ref) < 1e-3 and abs(prob[q] - ref_p) < 1e-3, (q, lg[q], ref)
    cts = [H.helrm_encrypt_query(ctx, evk, model, dense[q], idx[q], 7 + 3 * q) for q in range(3)]
    assert all(len(cs) == 2 for _, cs in cts)
    one = [H.helrm_infer_multi(ctx, evk, model, cd, cs) for cd, cs in cts]
    assert [H.helrm_decrypt_logit(ctx, sk, y)[0] for y in one] == list(lg)
    batch = H.helrm_batch_create(ctx, model, [evk] * 3)
    for y1, yb in zip(one, H.helrm_infer_batch(ctx, batch, [cd for cd, _ in cts], [cs for _, cs in cts])):
        (a, la, sa), (b, lb, sb) = H.helrm_ct_export(ctx, y1), H.helrm_ct_export(ctx, yb)
        assert la == lb and sa == sb and np.array_equal(a, b), "batched ciphertext differs"
    H.helrm_batch_set_graph(ctx, batch, True)    # capture, then replay
    for _ in range(2):
        ys = H.helrm_infer_batch(ctx, batch, [cd for cd, _ in cts], [x for _, cs in cts for x in cs])
        for y1, yg in zip(one, ys):
            (a, la, sa), (b, lb, sb) = H.helrm_ct_export(ctx, y1), H.helrm_ct_export(ctx, yg)
            assert la == lb and sa == sb and np.array_equal(a, b), "graph-replayed ciphertext differs"
    with pytest.raises(H.HelrmError) as e:      # one selector ciphertext is not the whole query
        H.helrm_infer(ctx, evk, model, cts[0][0], cts[0][1][0])
    assert e.value.name == "HELRM_E_INVAL"

    # the oracle's integer plaintexts and the same seeds: bit-exact
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    _, keys_o = ckks.keygen(p, 1, rot_steps=c.rotation_steps())
    xd, xs = dlrm.query_slots(p, c, dense[1], idx[1])
    assert len(xs) == 2
    md = ckks.encode_real(p, xd, p.delta)
    ms = [ckks.encode_real(p, x, p.delta) for x in xs]
    cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 300)
    cs = [H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, c.lvl_sel, p.delta), 301 + k) for k, m in enumerate(ms)]
    out_o = dlrm.infer(p, keys_o, c, ckks.encrypt(p, keys_o, md, c.lvl_dense, p.delta, 300),
                       [ckks.encrypt(p, keys_o, m, c.lvl_sel, p.delta, 301 + k) for k, m in enumerate(ms)])
    assert_ct_equal(ctx, H.helrm_infer_multi(ctx, evk, model, cd, cs), out_o)


def test_three_ciphertext_lookup_and_dlrm_share_giant_steps():
    """Three selector ciphertexts, the first two of one shape, so their
    products share one set of giant steps, ModDown, rescale and folds
    (reading R31).  The lookup at N = 2^12 (tables of 3000 and 1500 rows:
    2048 + 2048 + 404 columns) and the wider DLRM at N = 2^10 (1127 slots:
    512 + 512 + 103), one query and a lockstep batch of two, bit-exact
    against the oracle with its integer plaintexts."""
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 3)
    p = oracle_params(pr)
    cards, base = [3000, 1500], 4096
    rng = np.random.default_rng(32)
    tables = [[rng.uniform(-0.05, 0.05, (k, 16)).astype(np.float32)] for k in cards]
    ctx = gpu_ctx(pr)
    emb = H.helrm_emb_prepare(ctx, cards, base, 0, 16, tables, 0, 32, 2, p.delta, p.delta)
    assert H.helrm_emb_chunks(ctx, emb) == 3
    M = dlrm.embedding_matrix(cards, base, tables, 0, 32)
    pms = dlrm.prepare_multi(p, M, 32, 2, p.delta, p.delta)
    assert dlrm.lookup_groups(pms) == [[0, 1], [2]]
    mats = [H.helrm_emb_matrix(ctx, emb, c) for c in range(3)]
    steps = sorted(set().union(*[set(H.helrm_ptmat_rotations(ctx, m)) for m in mats]))
    sk, evk = H.helrm_keygen(ctx, 18, steps)
    _, keys_o = ckks.keygen(p, 18, rot_steps=steps, relin=False)
    for c in range(3):
        H.helrm_ptmat_import(ctx, mats[c], np.stack([pms[c].pts[k] for k in pms[c].ordered_keys()]).astype(np.int64))
    sel = dlrm.selector_vector(cards, base, (2999, 1499))
    ms = [ckks.encode_real(p, xi, p.delta) for xi in dlrm.chunk_slots(sel, p.n)]
    cts = [H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, 2, p.delta), 70 + c) for c, m in enumerate(ms)]
    cts_o = [ckks.encrypt(p, keys_o, m, 2, p.delta, 70 + c) for c, m in enumerate(ms)]
    y = H.helrm_embedding_lookup_multi(ctx, evk, emb, cts)
    assert_ct_equal(ctx, y, dlrm.lookup_multi(p, keys_o, pms, cts_o))
    want = np.concatenate(dlrm.embedding_cleartext(cards, base, tables, (2999, 1499)))
    assert np.max(np.abs(H.helrm_decrypt(ctx, sk, y, 32) - want)) < 1e-3

    pr = syn.reduced_params(10, 5)
    p = oracle_params(pr)
    spec = syn.wider_spec()
    w = syn.make_weights(spec, 0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    c = dlrm.compile_model(p, spec, w)
    assert H.helrm_model_info(ctx, model)["n_sel"] == c.n_sel() == 3
    assert dlrm.lookup_groups(c.emb_chunks) == [[0, 1], [2]]
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    steps = H.helrm_model_rotations(ctx, model)
    assert steps == c.rotation_steps()
    sk, evk = H.helrm_keygen(ctx, 3, steps)
    _, keys_o = ckks.keygen(p, 3, rot_steps=steps)
    dense, idx = syn.make_queries(spec, 1, seed=8)
    xd, xs = dlrm.query_slots(p, c, dense[0], idx[0])
    md = ckks.encode_real(p, xd, p.delta)
    msel = [ckks.encode_real(p, x, p.delta) for x in xs]
    cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 400)
    cs = [H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, c.lvl_sel, p.delta), 401 + k) for k, m in enumerate(msel)]
    out_o = dlrm.infer(p, keys_o, c, ckks.encrypt(p, keys_o, md, c.lvl_dense, p.delta, 400),
                       [ckks.encrypt(p, keys_o, m, c.lvl_sel, p.delta, 401 + k) for k, m in enumerate(msel)])
    assert_ct_equal(ctx, H.helrm_infer_multi(ctx, evk, model, cd, cs), out_o)
    batch = H.helrm_batch_create(ctx, model, [evk, evk])
    for yb in H.helrm_infer_batch(ctx, batch, [cd, cd], [cs, cs]):
        assert_ct_equal(ctx, yb, out_o)
    lg, _ = H.helrm_infer_e2e(ctx, sk, evk, model, dense, idx, 9)
    assert abs(lg[0] - dlrm.dlrm_cleartext(spec, w, dense[0], idx[0])[0]) < 1e-3
