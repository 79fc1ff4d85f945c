"""Bit-exact parity against the oracle at the full parameter set (N = 2^16,
q_0 60-bit + 20 x 40-bit, K = 3 x 60-bit special primes, alpha = 3).

The fixed-size NTT instances, which carry the fused base conversion, the
merged ModDown + rescale and the ModDown epilogue, run only at this ring
degree, as do the launch shapes the autotuner picks for it.  So the
key-switching operations are compared here word for word, on the same keys
and encryption randomness: rotations near the top of the chain, at the
embedding lookup's level and at level 1; hoisted rotations; a relinearised
product and a square; a degree-3 polynomial (products with the rescale
merged into the ModDown); and two BSGS matvecs at the lookup's level (a
square one with two giant steps, a wide one with a radix-4 fold level).
The oracle generates 18 keys at N = 2^16 (about a minute of host time).

Last, one UCI-shaped inference end to end at this size, through the path the
benchmark times (the server path of a batch of one, captured as a CUDA graph
and replayed): its logit ciphertext against the oracle's, word for word.  Its
47 oracle keys are made by the oracle's own key functions in a spawn-started
process pool, one key per task."""
import numpy as np
import pytest

from helpers import assert_ct_equal, gpu_ctx, oracle_keys_pool, oracle_params

pytestmark = pytest.mark.gpu

LOOKUP_LEVEL = 6
MATS = [(32, 32), (8, 32)]      # (rows, cols): D = 32 with n1 = 16, n2 = 2; D = 8 with folds 8, 16, 24


@pytest.fixture(scope="module")
def full():
    from oracle import ckks, linear
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]
    ctx, p = gpu_ctx(pr), oracle_params(pr)
    rng = np.random.default_rng(2024)
    mats = []
    for rows, cols in MATS:
        W = rng.normal(0, 0.3, (rows, cols))
        ip, op = linear.pow2ceil(cols), linear.pow2ceil(rows)
        mats.append((W, ip, op, linear.prepare(p, W, ip, op, LOOKUP_LEVEL, p.delta, p.delta)))
    steps = sorted({1, 5} | {s for *_, pm in mats for s in linear.rotation_steps(pm)})
    sk, evk = H.helrm_keygen(ctx, 61, steps)
    sk_o, keys_o = ckks.keygen(p, 61, rot_steps=steps, relin=True)
    return ctx, p, sk, evk, keys_o, steps, mats


def _fresh(full, level, seed):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, _, evk, keys_o = full[:5]
    z = np.random.default_rng(seed).uniform(-1, 1, p.n)
    m = ckks.encode_real(p, z, p.delta)
    return (H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, level, p.delta), seed),
            ckks.encrypt(p, keys_o, m, level, p.delta, seed), z)


def test_full_rotations(full):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk, keys_o, steps = full[:6]
    for level, step in [(18, 1), (LOOKUP_LEVEL, 5), (LOOKUP_LEVEL, steps[-1]), (1, 16)]:
        ct, ct_o, z = _fresh(full, level, 100 + level)
        r = H.helrm_rotate(ctx, evk, ct, step)
        assert_ct_equal(ctx, r, ckks.rotate(p, keys_o, ct_o, step))
        # the ModDown's uncorrected fast base conversion leaves a rounding error
        # of mean -u - 1/2 (u in [0, K)) per coefficient; times s, at N = 2^16,
        # it puts about 3.5e-6 into slot 0 (the oracle shows the same), 8e-8 elsewhere
        assert np.max(np.abs(H.helrm_decrypt(ctx, sk, r, 64) - np.roll(z, -step)[:64])) < 1e-5


def test_full_hoisted_rotations(full):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, _, evk, keys_o = full[:5]
    hs = [1, 5, 16, 0]
    ct, ct_o, _ = _fresh(full, LOOKUP_LEVEL, 120)
    want = ckks.rotate_hoisted(p, keys_o, ct_o, hs)
    for s, o in zip(hs, H.helrm_rotate_hoisted(ctx, evk, ct, hs)):
        assert_ct_equal(ctx, o, want[s])


def test_full_products_and_polynomial(full):
    from oracle import ckks, poly
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk, keys_o = full[:5]
    a, a_o, x = _fresh(full, 18, 130)
    b, b_o, y = _fresh(full, 18, 131)
    c = H.helrm_mul(ctx, evk, a, b)
    assert_ct_equal(ctx, c, ckks.mul(p, keys_o, a_o, b_o))
    assert np.max(np.abs(H.helrm_decrypt(ctx, sk, c, 64) - (x * y)[:64])) < 1e-5
    assert_ct_equal(ctx, H.helrm_mul(ctx, evk, a, a), ckks.square(p, keys_o, a_o))
    coeffs = (0.25, -1.0, 0.5, 0.125)
    yp = H.helrm_poly_eval(ctx, evk, a, coeffs, p.delta)
    assert_ct_equal(ctx, yp, poly.poly_eval(p, keys_o, a_o, coeffs, p.delta))
    got = H.helrm_decrypt(ctx, sk, yp, 64)
    assert np.max(np.abs(got - np.polynomial.polynomial.polyval(x[:64], np.asarray(coeffs)))) < 1e-4


@pytest.mark.parametrize("which", range(len(MATS)))
def test_full_matvec(full, which):
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk, keys_o = full[:5]
    W, ip, op, pm_o = full[6][which]
    pm = H.helrm_ptmat_prepare(ctx, W, ip, op, LOOKUP_LEVEL, p.delta, p.delta)
    info = H.helrm_ptmat_info(ctx, pm)
    assert (info["D"], info["n1"], info["n2"]) == (pm_o.layout.D, pm_o.layout.n1, pm_o.layout.n2)
    H.helrm_ptmat_import(ctx, pm, np.stack([pm_o.pts[k] for k in pm_o.ordered_keys()]).astype(np.int64))
    x = np.random.default_rng(140 + which).uniform(-1, 1, W.shape[1])
    m = ckks.encode_real(p, dlrm.replicate(x, ip, p.n), p.delta)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, LOOKUP_LEVEL, p.delta), 150 + which)
    ct_o = ckks.encrypt(p, keys_o, m, LOOKUP_LEVEL, p.delta, 150 + which)
    out = H.helrm_ptct_matvec(ctx, evk, pm, ct)
    assert_ct_equal(ctx, out, linear.matvec(p, keys_o, pm_o, ct_o))
    want = linear.matvec_cleartext(W, x, ip, op, p.n)
    assert np.max(np.abs(H.helrm_decrypt(ctx, sk, out, 256) - want[:256])) < 1e-3


def test_full_uci_inference_graph_bit_exact():
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]
    p = oracle_params(pr)
    spec = syn.uci_spec(0)
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    steps = c.rotation_steps()
    _, keys_o = oracle_keys_pool(pr, 77, steps)           # the pool starts before this test's first GPU call
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    assert H.helrm_model_rotations(ctx, model) == steps
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    sk, evk = H.helrm_keygen(ctx, 77, steps)
    batch = H.helrm_batch_create(ctx, model, [evk])
    H.helrm_batch_set_graph(ctx, batch, True)
    dense, idx = syn.make_queries(spec, 2, seed=33)
    for q in range(2):                                # the capture, then a replay
        xd, xs = dlrm.query_slots(p, c, dense[q], idx[q])
        md, ms = ckks.encode_real(p, xd, p.delta), ckks.encode_real(p, xs, p.delta)
        cd = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 40 + 2 * q)
        cs = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, c.lvl_sel, p.delta), 41 + 2 * q)
        y = H.helrm_infer_batch(ctx, batch, [cd], [cs])[0]
        if q == 1:
            y_o = dlrm.infer(p, keys_o, c, ckks.encrypt(p, keys_o, md, c.lvl_dense, p.delta, 40 + 2 * q),
                             ckks.encrypt(p, keys_o, ms, c.lvl_sel, p.delta, 41 + 2 * q))
            assert_ct_equal(ctx, y, y_o)
            lg = H.helrm_decrypt_logit(ctx, sk, y)[0]
            assert abs(lg - dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]) < 1e-3
