"""Edge cases of the lookup path on the GPU: tables at the digit boundaries
(1 row; exactly p rows, kept plain; p + 1; exactly p^2; p^2 + 1) looked up
at their first and last rows, bit-exact against the oracle and within 1e-3
of the gathered rows; the compression threshold at its boundary; empty
launches and batches."""
import numpy as np
import pytest

from helpers import assert_ct_equal, gpu_ctx, oracle_params

pytestmark = pytest.mark.gpu


def test_boundary_tables_bit_exact_and_accurate():
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 3)
    p = oracle_params(pr)
    cards, base = [1, 4, 5, 16, 17], 4
    rng = np.random.default_rng(71)
    tables = [[rng.uniform(-0.05, 0.05, (r, 16)).astype(np.float32) for r in syn.table_rows(k, base)]
              for k in cards]
    assert [len(t) for t in tables] == [1, 1, 2, 2, 3]
    ctx = gpu_ctx(pr)
    out_pad = 128                                     # 5 tables x 16 outputs, padded
    emb = H.helrm_emb_prepare(ctx, cards, base, 0, 16, tables, 0, out_pad, 2, p.delta, p.delta)
    width, period = H.helrm_emb_info(ctx, emb)
    assert (width, period) == (1 + 4 + 8 + 8 + 12, 64)
    M = dlrm.embedding_matrix(cards, base, tables, 0, out_pad)
    pm = linear.prepare(p, M, 64, out_pad, 2, p.delta, p.delta)
    steps = linear.rotation_steps(pm)
    assert sorted(H.helrm_ptmat_rotations(ctx, H.helrm_emb_matrix(ctx, emb, 0))) == sorted(steps)
    sk, evk = H.helrm_keygen(ctx, 73, steps)
    _, keys_o = ckks.keygen(p, 73, rot_steps=steps, relin=False)
    cases = [[0] * 5, [k - 1 for k in cards], [0, 3, 4, 15, 16], [0, 0, 4, 0, 8]]
    for idx in cases:                                # the library's own diagonals
        sel = dlrm.replicate(dlrm.selector_vector(cards, base, idx), 64, p.n)
        assert np.array_equal(H.helrm_query_pack(ctx, emb, idx, p.n), sel)
        ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, sel, 2, p.delta), 80)
        got = H.helrm_decrypt(ctx, sk, H.helrm_embedding_lookup(ctx, evk, emb, ct), 80)
        want = np.concatenate(dlrm.embedding_cleartext(cards, base, tables, idx))
        assert np.max(np.abs(got - want)) < 1e-3, idx
    # the oracle's integer diagonals and the same encryption: bit for bit
    H.helrm_ptmat_import(ctx, H.helrm_emb_matrix(ctx, emb, 0),
                         np.stack([pm.pts[k] for k in pm.ordered_keys()]).astype(np.int64))
    m = ckks.encode_real(p, dlrm.replicate(dlrm.selector_vector(cards, base, cases[1]), 64, p.n), p.delta)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, 2, p.delta), 81)
    assert_ct_equal(ctx, H.helrm_embedding_lookup(ctx, evk, emb, ct),
                    linear.matvec(p, keys_o, pm, ckks.encrypt(p, keys_o, m, 2, p.delta, 81)))


def test_threshold_boundary_layout():
    """A table with as many rows as the threshold stays a plain one-hot; one
    row more is digit-decomposed (base 2: 4 digits for 9 rows)."""
    from oracle import dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 3)
    ctx = gpu_ctx(pr)
    cards, base, thr = [8, 9], 2, 8
    rng = np.random.default_rng(3)
    tables = [[rng.uniform(-0.05, 0.05, (r, 16)).astype(np.float32) for r in syn.table_rows(k, base, thr)]
              for k in cards]
    emb = H.helrm_emb_prepare(ctx, cards, base, thr, 16, tables, 0, 32, 2, 2.0**40, 2.0**40)
    lay, w = dlrm.selector_layout(cards, base, thr)
    assert H.helrm_emb_info(ctx, emb)[0] == w == 8 + 4 * 2
    for idx in ([7, 8], [0, 0], [3, 5]):
        n = H.helrm_ctx_dims(ctx)[1]
        assert np.array_equal(H.helrm_query_pack(ctx, emb, idx, n),
                              dlrm.replicate(dlrm.selector_vector(cards, base, idx, thr), 16, n))


def test_empty_launches_and_batches():
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 9)
    ctx = gpu_ctx(pr)
    buf = torch.zeros(8, dtype=torch.int64, device="cuda")
    H.helrm_ntt(ctx, buf.data_ptr(), 0, 1, False)                 # zero limbs: nothing to do
    H.helrm_ctx_synchronize(ctx)
    spec = syn.uci_spec(0)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    with pytest.raises(H.HelrmError) as e:                        # a batch of no queries
        H.helrm_batch_create(ctx, model, [])
    assert e.value.name == "HELRM_E_INVAL"
    sk, evk = H.helrm_model_keygen(ctx, model, 4)
    lg, _ = H.helrm_infer_e2e(ctx, sk, evk, model, np.zeros((0, spec.n_dense)), np.zeros((0, 8), np.int64), 1)
    assert len(lg) == 0                                           # no queries: no logits
