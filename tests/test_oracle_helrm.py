"""Pins for the HE-LRM layer of the oracle: digit decomposition, selectors,
block-diagonal packing, the BSGS matvec, the encrypted lookup, and the
encrypted DLRM against the FP64 cleartext model."""
import json
import os

import numpy as np
import pytest

from oracle import ckks, dlrm, linear
from paper_2506_18150_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_digit_decomposition_paper_example():
    g = json.load(open(os.path.join(GOLDEN, "digit_example.json")))
    assert dlrm.num_digits(g["k"], g["p"]) == g["ell"]
    assert dlrm.digits(g["i"], g["p"], g["ell"]) == g["digits"]


def test_digits_reconstruct_every_index():
    for k, p in [(16, 4), (1024, 32), (10**7, 64), (65, 64), (64, 64)]:
        ell = dlrm.num_digits(k, p)
        assert p**ell >= k and (ell == 1 or p ** (ell - 1) < k)
        for i in list(range(min(k, 300))) + [k - 1]:
            d = dlrm.digits(i, p, ell)
            assert all(0 <= x < p for x in d) and sum(x * p**j for j, x in enumerate(d)) == i


def test_parameter_reduction_is_p_l_d():
    """O(kd) -> O(p l d) parameters (Sec. 4.1.1)."""
    k, p, d = 10**7, 64, 16
    assert sum(syn.table_rows(k, p)) * d == p * dlrm.num_digits(k, p) * d == 4096


def test_lookup_matrix_is_the_gather_for_all_1024_indices():
    C = syn.tiny_table(0)
    M = dlrm.lookup_matrix(C, 32, 1024)
    assert M.shape == (16, 64)
    for i in range(1024):
        sel = dlrm.selector_vector([1024], 32, [i])
        assert sel.sum() == 2 and sel[i % 32] == 1 and sel[32 + i // 32] == 1
        want = C[0][i % 32].astype(np.float64) + C[1][i // 32].astype(np.float64)
        assert np.allclose(M @ sel, want, atol=1e-12)


def test_block_diagonal_packing_gives_contiguous_outputs():
    spec = syn.uci_spec(0)
    w = syn.make_weights(spec, 0)
    _, idx = syn.make_queries(spec, 5, seed=1)
    M = dlrm.embedding_matrix(spec.cards, spec.base, w.tables, 16, 16 * 9)
    for q in range(5):
        y = M @ dlrm.selector_vector(spec.cards, spec.base, idx[q])
        embs = dlrm.embedding_cleartext(spec.cards, spec.base, w.tables, idx[q])
        assert np.allclose(y[:16], 0) and np.allclose(y[16:], np.concatenate(embs))


def test_uci_paper_packing_uses_28_slots():
    s = syn.uci_paper_spec()
    _, width = dlrm.selector_layout(s.cards, s.base)
    assert s.n_dense + width == 28


def test_selector_ciphertext_counts_and_compression_table():
    t = json.load(open(os.path.join(GOLDEN, "compression_table.json")))
    n = t["slots_per_ct"]
    for row in t["rows"]:
        if "cts" in row:
            assert -(-row["slots"] // n) == row["cts"]
        # CR x slots is the total row count of the uncompressed model (~33.8M)
        assert abs(row["cr"] * row["slots"] / t["total_rows"] - 1) < 0.02
    assert -(-int(t["total_rows"]) // n) == t["naive_cts"]


def test_diagonal_count_for_416_outputs():
    """26 tables x 16 = 416 outputs, padded to 512: 512 diagonals (Sec. 5.4)."""
    lay = linear.Layout.make(in_pad=8192, out_pad=linear.pow2ceil(416))
    assert lay.D == 512 and lay.n1 * lay.n2 == 512 and lay.folds == [(512, 4), (2048, 4)]
    assert linear.Layout.make(in_pad=512, out_pad=512).D == 512


def test_fold_plan_covers_every_offset_once():
    """The fold levels sum rot(y, j out_pad) for every j < in_pad / out_pad
    exactly once: the offsets sum_t d_t stride_t (d_t < radix_t) are
    0, out_pad, ..., in_pad - out_pad without repetition."""
    import itertools
    for out_pad in (1, 16, 512):
        for b in range(0, 13):
            in_pad = out_pad << b
            plan = linear.fold_plan(in_pad, out_pad)
            assert all(r <= 4 for _, r in plan) and len(plan) == (b + 1) // 2
            offs = [sum(d * s for d, (s, _) in zip(ds, plan))
                    for ds in itertools.product(*[range(r) for _, r in plan])]
            assert sorted(offs) == list(range(0, in_pad, out_pad))


def test_bsgs_split():
    for D, n1, n2 in [(1, 1, 1), (2, 2, 1), (16, 16, 1), (32, 16, 2), (64, 16, 4), (128, 16, 8),
                      (256, 32, 8), (512, 64, 8), (1024, 128, 8)]:
        assert linear.bsgs_split(D) == (n1, n2)
    for k in range(16):   # every power-of-two D: an exact split with at most 8 giant steps
        n1, n2 = linear.bsgs_split(1 << k)
        assert n1 * n2 == 1 << k and n2 <= 8


@pytest.mark.parametrize("shape", [(16, 64), (64, 16), (32, 32), (1, 32), (10, 3), (5, 7)])
def test_bsgs_matvec_matches_cleartext(small_params, shape):
    p = small_params
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    W = rng.normal(0, 0.3, shape)
    x = rng.uniform(-1, 1, shape[1])
    ip, op = linear.pow2ceil(shape[1]), linear.pow2ceil(shape[0])
    pm = linear.prepare(p, W, ip, op, 3, p.delta, p.delta)
    sk, keys = ckks.keygen(p, 55, rot_steps=linear.rotation_steps(pm), relin=False)
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, dlrm.replicate(x, ip, p.n), p.delta), 3, p.delta, 6)
    out = linear.matvec(p, keys, pm, ct)
    assert out.level == 2                                    # one level consumed
    got = ckks.decrypt(p, sk, out)
    assert np.max(np.abs(got - linear.matvec_cleartext(W, x, ip, op, p.n))) < 1e-5


@pytest.fixture(scope="module")
def tiny():
    pr = syn.PARAMS["tiny"]
    p = ckks.Params(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"])
    C = syn.tiny_table(0)
    M = dlrm.lookup_matrix(C, 32, 1024)
    pm = linear.prepare(p, M, 64, 16, 1, p.delta, p.delta)
    pm_d = [linear.prepare(p, M[:, 32 * j: 32 * j + 32], 32, 16, 1, p.delta, p.delta) for j in range(2)]
    steps = sorted(set(linear.rotation_steps(pm)) | set(linear.rotation_steps(pm_d[0])))
    sk, keys = ckks.keygen(p, 0, rot_steps=steps, relin=False)
    return p, C, M, pm, pm_d, sk, keys


def test_tiny_lookup_packed_and_separate(tiny):
    """Config 'tiny': 1024 x 16 table in base 32; (a) both digit selectors in one
    ciphertext (64 slots), (b) each selector its own ciphertext (sum of two
    matvecs).  Decrypted row vs the cleartext gather, max-abs <= 1e-3."""
    p, C, M, pm, pm_d, sk, keys = tiny
    rng = np.random.default_rng(0)
    for i in rng.integers(0, 1024, 3):
        want = C[0][i % 32].astype(np.float64) + C[1][i // 32].astype(np.float64)
        sel = dlrm.selector_vector([1024], 32, [i])
        ct = ckks.encrypt(p, keys, ckks.encode_real(p, dlrm.replicate(sel, 64, p.n), p.delta), 1, p.delta, int(i))
        out = linear.matvec(p, keys, pm, ct)
        assert out.level == 0
        got = ckks.decrypt(p, sk, out)
        assert np.max(np.abs(got[:16] - want)) < 1e-3
        assert np.max(np.abs(got - np.tile(want, p.n // 16))) < 1e-3
        parts = []
        for j in range(2):
            s = dlrm.replicate(sel[32 * j: 32 * j + 32], 32, p.n)
            c = ckks.encrypt(p, keys, ckks.encode_real(p, s, p.delta), 1, p.delta, int(i) + 7 * j)
            parts.append(linear.matvec(p, keys, pm_d[j], c))
        got2 = ckks.decrypt(p, sk, ckks.add(p, parts[0], parts[1]))
        assert np.max(np.abs(got2[:16] - want)) < 1e-3


@pytest.mark.parametrize("interaction", ["dot", "concat"])
def test_encrypted_uci_dlrm_matches_cleartext(interaction):
    spec = syn.uci_spec(0, interaction)
    w = syn.make_weights(spec, 0)
    pr = syn.reduced_params(13, 9)
    p = ckks.Params(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"])
    c = dlrm.compile_model(p, spec, w)
    assert (c.lvl_dense, c.lvl_sel) == ((9, 6) if interaction == "dot" else (7, 4))
    sk, keys = ckks.keygen(p, 1, rot_steps=c.rotation_steps())
    dense, idx = syn.make_queries(spec, 1, seed=5)
    cd, cs = dlrm.encrypt_query(p, keys, c, dense[0], idx[0], 100)
    out = dlrm.infer(p, keys, c, cd, cs)
    assert out.level == 0
    logit, prob = dlrm.decrypt_logit(p, sk, out)
    ref, ref_prob, _ = dlrm.dlrm_cleartext(spec, w, dense[0], idx[0])
    assert abs(logit - ref) < 1e-3 and abs(prob - ref_prob) < 1e-3


def test_criteo_shape():
    spec = syn.criteo_spec(0)
    assert len(spec.cards) == 26 and abs(sum(spec.cards) / 33.8e6 - 1) < 0.005
    assert min(spec.cards) >= 3 and max(spec.cards) <= 10**7
    assert spec.top[0] == 16 + 27 * 26 // 2 == 367
    _, width = dlrm.selector_layout(spec.cards, spec.base)
    assert 2048 < width <= 8192
    assert syn.uci_spec(0).top[0] == 52


def test_selector_chunks_cover_the_width_once():
    """Selectors wider than n slots split into ceil(width / n) ciphertexts."""
    for width, n in [(560, 512), (512, 512), (1, 512), (33_000, 32_768), (2_772_109, 32_768)]:
        ch = dlrm.selector_chunks(width, n)
        assert len(ch) == -(-width // n)
        assert [c0 for c0, _ in ch] == list(range(0, width, n))
        assert sum(w for _, w in ch) == width and all(0 < w <= n for _, w in ch)
    assert len(dlrm.selector_chunks(2_772_109, 32_768)) == 85        # Sec. 5.4: the 12.18x model


def test_two_ciphertext_lookup_has_1024_diagonals():
    """416 outputs (padded to 512) over a selector spanning two ciphertexts of
    n = 2^15 slots: 512 diagonals per ciphertext, 1024 in all (Sec. 5.4)."""
    n = 1 << 15
    chunks = dlrm.selector_chunks(n + 5000, n)
    lays = [linear.Layout.make(linear.pow2ceil(w), linear.pow2ceil(416)) for _, w in chunks]
    assert len(lays) == 2 and sum(l.D for l in lays) == 1024


def test_multi_ciphertext_lookup_matches_gather(small_params):
    """N = 2^10 (n = 512 slots): two plain tables of 300 and 260 rows give a
    560-slot selector, i.e. two ciphertexts (512 + 48 columns).  The sum of the
    two per-ciphertext BSGS products decrypts to the gathered embeddings."""
    p = small_params
    cards, base = [300, 260], 512
    rng = np.random.default_rng(12)
    tables = [[rng.uniform(-0.05, 0.05, (k, dlrm.DIM)).astype(np.float32)] for k in cards]
    M = dlrm.embedding_matrix(cards, base, tables, 0, 2 * dlrm.DIM)
    pms = dlrm.prepare_multi(p, M, 2 * dlrm.DIM, 3, p.delta, p.delta)
    assert [pm.layout.in_pad for pm in pms] == [512, 64]
    steps = sorted(set().union(*[linear.rotation_steps(pm) for pm in pms]))
    sk, keys = ckks.keygen(p, 21, rot_steps=steps, relin=False)
    for idx in [(0, 0), (299, 259), (17, 200)]:
        sel = dlrm.selector_vector(cards, base, idx)
        x = dlrm.chunk_slots(sel, p.n)
        # the block decomposition in the clear: M s = sum_c M_c s_c
        parts = [M[:, c0:c0 + w] @ sel[c0:c0 + w] for c0, w in dlrm.selector_chunks(len(sel), p.n)]
        assert np.allclose(sum(parts), M @ sel)
        cts = [ckks.encrypt(p, keys, ckks.encode_real(p, xi, p.delta), 3, p.delta, 40 + c) for c, xi in enumerate(x)]
        y = dlrm.lookup_multi(p, keys, pms, cts)
        assert y.level == 2
        got = ckks.decrypt(p, sk, y)[: 2 * dlrm.DIM]
        want = np.concatenate(dlrm.embedding_cleartext(cards, base, tables, idx))
        assert np.max(np.abs(got - want)) < 1e-4, idx


def test_multi_ciphertext_lookup_shares_giant_steps(small_params):
    """Three selector ciphertexts (plain tables of 600 and 500 rows at n = 512
    slots: 512 + 512 + 76 columns): the two full chunks have the same shape
    and share one set of giant steps, ModDown, rescale and folds
    (linear.matvec_sum, reading R31).  The lookup decrypts to the gathered
    rows; a one-matrix matvec_sum is matvec word for word; and the shared
    tail decrypts to the sum of the two separate products."""
    p = small_params
    cards, base = [600, 500], 1024
    rng = np.random.default_rng(13)
    tables = [[rng.uniform(-0.05, 0.05, (k, dlrm.DIM)).astype(np.float32)] for k in cards]
    M = dlrm.embedding_matrix(cards, base, tables, 0, 2 * dlrm.DIM)
    pms = dlrm.prepare_multi(p, M, 2 * dlrm.DIM, 3, p.delta, p.delta)
    assert [pm.layout.in_pad for pm in pms] == [512, 512, 128]
    assert dlrm.lookup_groups(pms) == [[0, 1], [2]]
    steps = sorted(set().union(*[linear.rotation_steps(pm) for pm in pms]))
    sk, keys = ckks.keygen(p, 22, rot_steps=steps, relin=False)
    idx = (599, 3)
    sel = dlrm.selector_vector(cards, base, idx)
    cts = [ckks.encrypt(p, keys, ckks.encode_real(p, xi, p.delta), 3, p.delta, 50 + c)
           for c, xi in enumerate(dlrm.chunk_slots(sel, p.n))]
    y = dlrm.lookup_multi(p, keys, pms, cts)
    got = ckks.decrypt(p, sk, y)[: 2 * dlrm.DIM]
    want = np.concatenate(dlrm.embedding_cleartext(cards, base, tables, idx))
    assert np.max(np.abs(got - want)) < 1e-4
    one, alone = linear.matvec_sum(p, keys, [pms[2]], [cts[2]]), linear.matvec(p, keys, pms[2], cts[2])
    assert np.array_equal(one.c0, alone.c0) and np.array_equal(one.c1, alone.c1)
    both = linear.matvec_sum(p, keys, pms[:2], cts[:2])
    sep = ckks.add(p, linear.matvec(p, keys, pms[0], cts[0]), linear.matvec(p, keys, pms[1], cts[1]))
    assert not np.array_equal(both.c0, sep.c0)          # a different rounding path ...
    assert np.max(np.abs(ckks.decrypt(p, sk, both) - ckks.decrypt(p, sk, sep))) < 1e-5   # ... to the same sum
    with pytest.raises(ValueError):
        linear.matvec_sum(p, keys, [pms[0], pms[2]], [cts[0], cts[2]])


def test_threshold_policy_layout():
    """Sec. 5.2's policy: a table is digit-decomposed (base p) only if it has
    more rows than the threshold; with the threshold at p this is the plain
    rule (a table that fits one digit stays a plain one-hot)."""
    cards = [700, 2000, 3]
    lay, w = dlrm.selector_layout(cards, 4, 1000)
    assert [(t, j, ww) for (t, j, _, ww) in lay] == [(0, 0, 700)] + [(1, j, 4) for j in range(6)] + [(2, 0, 3)]
    assert w == 700 + 6 * 4 + 3 == 727
    assert dlrm.selector_layout(cards, 4, None) == dlrm.selector_layout(cards, 4, 4)
    # uncompressed everything: one slot per row, CR = 1
    assert dlrm.selector_layout(cards, 4, 10**9)[1] == sum(cards)
    # slots as a function of the threshold (the paper's CR = rows / slots)
    for thr in [3, 700, 1000, 2000]:
        want = sum(k if k <= thr else 4 * dlrm.num_digits(k, 4) for k in cards)
        assert dlrm.selector_layout(cards, 4, thr)[1] == want
    s = syn.wide_spec()
    assert [sum(syn.table_rows(k, s.base, s.threshold)) for k in s.cards] == [700, 24, 3]
    rng = np.random.default_rng(4)
    w_ = syn.make_weights(s, 0)
    for _ in range(20):
        idx = [int(rng.integers(0, k)) for k in cards]
        M = dlrm.embedding_matrix(cards, 4, w_.tables, 0, 48, threshold=1000)
        y = M @ dlrm.selector_vector(cards, 4, idx, 1000)
        assert np.allclose(y, np.concatenate(dlrm.embedding_cleartext(cards, 4, w_.tables, idx, 1000)))


def test_encrypted_dlrm_with_two_selector_ciphertexts(small_params):
    """N = 2^10 (512 slots): the wide model's 727-slot selector spans two
    ciphertexts; the encrypted logit (lookup = sum of the two per-ciphertext
    products) matches the FP64 cleartext DLRM."""
    p = small_params
    spec = syn.wide_spec()
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    assert c.emb is None and c.n_sel() == 2
    assert [pm.layout.in_pad for pm in c.emb_chunks] == [512, 256]
    sk, keys = ckks.keygen(p, 8, rot_steps=c.rotation_steps())
    dense, idx = syn.make_queries(spec, 2, seed=6)
    for q in range(2):
        cd, cs = dlrm.encrypt_query(p, keys, c, dense[q], idx[q], 200 + 3 * q)
        assert len(cs) == 2
        out = dlrm.infer(p, keys, c, cd, cs)
        logit, _ = dlrm.decrypt_logit(p, sk, out)
        ref = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]
        assert abs(logit - ref) < 1e-3, (q, logit, ref)


def test_encrypted_dlrm_with_polynomial_silu():
    """A tiny DLRM (bottom 4-16, tables of 3 and 5 rows, dot interaction, top
    19-1) whose activation is the degree-6 SiLU polynomial: the activation
    costs poly.depth(6) = 4 levels, so ct_dense sits at level 3 + 5 = 8, and
    the encrypted logit matches the FP64 DLRM with the same polynomial."""
    from oracle import poly
    p = ckks.Params(10, [60] + [40] * 8, 3, 60, 3, 40.0)
    spec = syn.DLRMSpec("tiny_silu", 4, [4, 16], [0, 1], [3, 5], 8, 16, "dot", act=syn.silu_poly(7))
    spec.top[0] = syn.top_input_width(spec)
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    assert dlrm.activation_levels(spec) == poly.depth(6) == 4
    assert (c.lvl_dense, c.lvl_sel, c.lvl_z, c.lvl_u) == (8, 4, 3, 1)
    sk, keys = ckks.keygen(p, 8, rot_steps=c.rotation_steps())
    dense, idx = syn.make_queries(spec, 2, seed=3)
    for q in range(2):
        cd, cs = dlrm.encrypt_query(p, keys, c, dense[q], idx[q], 60 + 3 * q)
        logit, _ = dlrm.decrypt_logit(p, sk, dlrm.infer(p, keys, c, cd, cs))
        ref = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]
        assert abs(logit - ref) < 1e-3, (q, logit, ref)
