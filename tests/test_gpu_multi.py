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
    emb = H.helrm_emb_prepare(ctx, cards, base, 16, tables, 0, 32, 2, p.delta, p.delta)
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
