"""Bootstrapping on the GPU (Sec. 2.1.4, Sec. 5.4) against the oracle
(oracle/boot.py): every stage word for word (ModRaise, SubSum, CoeffToSlot,
EvalMod, SlotToCoeff) with the oracle's diagonals and cosine polynomial
imported, on the bootstrappable chain at small N; the library's own
constants next to the oracle's; and the refreshed message at the full
parameter set (N = 2^16, n_s = 512, the Criteo models' widest layer)."""
import numpy as np
import pytest

from helpers import assert_ct_equal, gpu_ctx, import_ct, oracle_params

pytestmark = pytest.mark.gpu

H_SECRET, SEED = 192, 7


def _oracle_setup(pr, n_s):
    from oracle import boot, ckks
    p = oracle_params(pr)
    b = boot.prepare(p, boot.BootParams(n_s=n_s))
    sk, keys = ckks.keygen(p, SEED, rot_steps=b.rotation_steps(), h=H_SECRET, conj=True)
    return p, b, sk, keys


def _gpu_boot(ctx, p, b_or):
    """The library's bootstrapping with the oracle's polynomial and diagonals imported."""
    from paper_2506_18150_gb300 import helrm as H
    bt = H.helrm_boot_create(ctx, b_or.bp.n_s, coeffs=b_or.coeffs)
    mats = [b_or.cts[0], b_or.stc]
    info = H.helrm_boot_info(ctx, bt)
    assert info["n_plaintexts"] == sum(len(pm.pts) for pm in mats)
    for w, pm in enumerate(mats):
        H.helrm_ptmat_import(ctx, H.helrm_boot_matrix(ctx, bt, w), np.stack([pm.pts[k] for k in pm.ordered_keys()]))
    return bt


@pytest.mark.parametrize("log_n,n_s", [(10, 64), (11, 256), (10, 4), (10, 1), (10, 256)])
def test_bootstrap_stages_bit_exact(log_n, n_s):
    from oracle import boot, ckks
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params(log_n, 4)
    p, b_or, sk_or, keys = _oracle_setup(pr, n_s)
    ctx = gpu_ctx(pr)
    bt = _gpu_boot(ctx, p, b_or)
    steps = H.helrm_boot_rotations(ctx, bt)
    assert steps == b_or.rotation_steps()
    sk, evk = H.helrm_keygen_ex(ctx, SEED, H_SECRET, steps, conj=True)
    z = np.random.default_rng(log_n + n_s).uniform(-1, 1, n_s)[np.arange(p.n) % n_s]
    ct_or = ckks.encrypt(p, keys, ckks.encode_real(p, z, p.delta), 2, p.delta, 11)
    st_or = {}
    out_or = boot.bootstrap(p, keys, b_or, ct_or, st_or)
    out, st = H.helrm_bootstrap(ctx, evk, bt, import_ct(ctx, ct_or), stages=True)
    for name, g in zip(["raised", "subsum", "cts", "evalmod", "out"], st):
        assert_ct_equal(ctx, g, st_or[name])
    assert_ct_equal(ctx, out, out_or)
    assert H.helrm_boot_info(ctx, bt)["level_out"] == out_or.level
    got = H.helrm_decrypt(ctx, sk, out, p.n)
    assert np.max(np.abs(got - z)) < 1e-6 + _sine_bound(p, b_or, z)


def _sine_bound(p, b_or, z):
    """EvalMod returns sin(2 pi u) / (2 pi) for u = 2^b m_k / q_0 on every
    coefficient m_k of the Delta-scaled message, u minus (2 pi)^2 u^3 / 6 to
    first order; a slot gathers the errors of all coefficients (|U| = 1).
    With n_s = 1 the one non-zero coefficient is z Delta itself, so the
    error is about 6e-6 z^3 at 2^b = 2^10 and a 60-bit q_0; with n_s = 64
    the coefficients are about z / 8 and the term vanishes."""
    from oracle import ckks
    m = ckks.encode_real(p, z, p.delta).astype(np.float64)
    u = m * 2.0**b_or.bp.log2_boost / float(p.q[0])
    return 1.05 * float(np.sum(np.abs(m / p.delta) * (2 * np.pi * u) ** 2 / 6))


def test_sparse_keys_and_conjugation_bit_exact():
    """The sparse secret and the conjugation key: an oracle ciphertext
    conjugated by both sides, and a GPU encryption under the sparse public
    key equal to the oracle's."""
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(11, 3)
    p = oracle_params(pr)
    ctx = gpu_ctx(pr)
    sk_or, keys = ckks.keygen(p, 23, rot_steps=[3], h=64, conj=True)
    sk, evk = H.helrm_keygen_ex(ctx, 23, 64, [3], conj=True)
    rng = np.random.default_rng(2)
    zc = rng.uniform(-1, 1, p.n) + 1j * rng.uniform(-1, 1, p.n)
    m = ckks.encode_complex(p, zc, p.delta)
    ct_or = ckks.encrypt(p, keys, m, 3, p.delta, 5)
    assert_ct_equal(ctx, H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, 3, p.delta), 5), ct_or)
    assert_ct_equal(ctx, H.helrm_conjugate(ctx, evk, import_ct(ctx, ct_or)), ckks.conjugate(p, keys, ct_or))
    assert_ct_equal(ctx, H.helrm_rotate(ctx, evk, import_ct(ctx, ct_or), 3), ckks.rotate(p, keys, ct_or, 3))
    # the dense default is helrm_keygen's
    _, evk0 = H.helrm_keygen_ex(ctx, 23, 0, [])
    _, evk1 = H.helrm_keygen(ctx, 23, [])
    pt = H.helrm_pt_import(ctx, m, 3, p.delta)
    a = H.helrm_ct_export(ctx, H.helrm_encrypt(ctx, evk0, pt, 9))[0]
    b = H.helrm_ct_export(ctx, H.helrm_encrypt(ctx, evk1, pt, 9))[0]
    assert np.array_equal(a, b)


def test_library_constants_next_to_the_oracle():
    """The library's own cosine fit and encoded diagonals (no import) against
    the oracle's: the two fits as functions within 1e-12 of each other and of
    cos(2 pi y) on the interval (their high power-basis coefficients differ in
    the last digits: the conversion from the Chebyshev basis cancels), the
    diagonals within one unit (the two FFT encoders round independently)."""
    from oracle import boot
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params(10, 4)
    p = oracle_params(pr)
    b_or = boot.prepare(p, boot.BootParams(n_s=64))
    ctx = gpu_ctx(pr)
    bt = H.helrm_boot_create(ctx, 64)
    cf = np.array(H.helrm_boot_coeffs(ctx, bt))
    want = np.array(b_or.coeffs)
    assert all(cf[1::2] == 0.0) and cf.shape == want.shape
    Y = (b_or.bp.K + 0.5) / 2.0**b_or.bp.r
    y = np.linspace(-Y, Y, 100001)
    pv = np.polynomial.polynomial.polyval
    assert np.max(np.abs(pv(y, cf) - pv(y, want))) < 1e-12
    assert np.max(np.abs(pv(y, cf) - np.cos(2 * np.pi * y))) < 1e-12
    for w, pm in enumerate([b_or.cts[0], b_or.stc]):
        got = H.helrm_ptmat_export(ctx, H.helrm_boot_matrix(ctx, bt, w), len(pm.pts), p.N)
        ref = np.stack([pm.pts[k] for k in pm.ordered_keys()])
        assert np.max(np.abs(got - ref)) <= 1, w


def test_boot_errors():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    ctx = gpu_ctx(syn.boot_params(10, 4))
    for kw, name in [(dict(n_s=3), "HELRM_E_INVAL"), (dict(n_s=512), "HELRM_E_INVAL"),
                     (dict(n_s=64, degree=15), "HELRM_E_INVAL"), (dict(n_s=64, r=12), "HELRM_E_PARAM")]:
        with pytest.raises(H.HelrmError) as e:
            H.helrm_boot_create(ctx, **kw)
        assert e.value.name == name, kw
    bt = H.helrm_boot_create(ctx, 64)
    sk, evk = H.helrm_keygen_ex(ctx, 3, 192, [])          # no rotation keys
    ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, np.zeros(64), 1, 2.0**40), 1)
    with pytest.raises(H.HelrmError) as e:
        H.helrm_bootstrap(ctx, evk, bt, ct)
    assert e.value.name == "HELRM_E_NOKEY"


def test_bootstrap_full_size_refreshes_the_message():
    """N = 2^16 on the bootstrappable chain (13 compute + 13 bootstrapping
    primes), n_s = 512, the library's own constants: the output is at level
    13 with the input's values within 1e-4 (measured: 1.3e-5; the sine's
    cubic term alone is up to 6.5e-6 for a unit message raised to 2^-10 of
    q_0, the rest is the noise the 6 double angles multiply by up to 4^6); a
    second bootstrap of the output (dropped to level 0) keeps them."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params()
    ctx = gpu_ctx(pr)
    n_s, n = 512, 1 << (pr["log_n"] - 1)
    bt = H.helrm_boot_create(ctx, n_s)
    info = H.helrm_boot_info(ctx, bt)
    assert (info["level_top"], info["level_out"]) == (26, 13)
    sk, evk = H.helrm_keygen_ex(ctx, 5, H_SECRET, H.helrm_boot_rotations(ctx, bt), conj=True)
    z = np.random.default_rng(9).uniform(-1, 1, n_s)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, z[np.arange(n) % n_s], 0, 2.0**40), 3)
    y = H.helrm_bootstrap(ctx, evk, bt, ct)
    lvl = H.helrm_ct_info(ctx, y)[0]
    assert lvl == 13
    got = H.helrm_decrypt(ctx, sk, y, n_s)
    assert np.max(np.abs(got - z)) < 1e-4
    y2 = H.helrm_bootstrap(ctx, evk, bt, H.helrm_drop_level(ctx, y, 0))
    assert np.max(np.abs(H.helrm_decrypt(ctx, sk, y2, n_s) - z)) < 2e-4


def test_bootstrapped_dlrm_bit_exact():
    """The UCI-shaped SiLU model (concatenation) with bootstraps before bottom
    layer 1 and on z, at N = 2^10 on the bootstrappable chain: with the
    oracle's plaintexts (the bootstraps' diagonals included) and cosine
    polynomial, the logit ciphertext of helrm_infer and of a batch of two
    equals the oracle's word for word, eagerly and replayed as a CUDA graph."""
    from oracle import boot, ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params(10, 10)
    p = oracle_params(pr)
    spec = syn.uci_silu_boot_spec(0)
    spec.boot_coeffs = tuple(boot.cos_fit(24, 6, 16))
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    info = H.helrm_model_info(ctx, model)
    assert (info["lvl_dense"], info["lvl_sel"]) == (c.lvl_dense, c.lvl_sel)
    pts = c.plaintexts()
    assert info["n_plaintexts"] == len(pts)
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in pts]))
    assert H.helrm_model_rotations(ctx, model) == c.rotation_steps()
    sk, evk = H.helrm_model_keygen(ctx, model, 3)
    _, keys = ckks.keygen(p, 3, rot_steps=c.rotation_steps(), h=H_SECRET, conj=True)
    dense, idx = syn.make_queries(spec, 2, seed=5)
    cts = [dlrm.encrypt_query(p, keys, c, dense[q], idx[q], 100 + 2 * q) for q in range(2)]
    want = [dlrm.infer(p, keys, c, cd, cs) for cd, cs in cts]
    for q, (cd, cs) in enumerate(cts):
        assert_ct_equal(ctx, H.helrm_infer(ctx, evk, model, import_ct(ctx, cd), import_ct(ctx, cs)), want[q])
    bt = H.helrm_batch_create(ctx, model, [evk, evk])
    ys = H.helrm_infer_batch(ctx, bt, [import_ct(ctx, cd) for cd, _ in cts], [import_ct(ctx, cs) for _, cs in cts])
    for q in range(2):
        assert_ct_equal(ctx, ys[q], want[q])
    H.helrm_batch_set_graph(ctx, bt, True)
    for _ in range(2):                                  # the capture, then a replay
        ys = H.helrm_infer_batch(ctx, bt, [import_ct(ctx, cd) for cd, _ in cts], [import_ct(ctx, cs) for _, cs in cts])
        for q in range(2):
            assert_ct_equal(ctx, ys[q], want[q])
    logit = H.helrm_decrypt_logit(ctx, sk, ys[0])[0]
    assert abs(logit - dlrm.dlrm_cleartext(spec, w, dense[0], idx[0])[0]) < 1e-4


def test_served_bootstrapped_dlrm_bit_exact():
    """The bootstrapped UCI-shaped SiLU model (N = 2^10) through the serving
    loop: a burst of three requests of one client batched together; every
    served logit ciphertext equals the oracle's dlrm.infer word for word."""
    from oracle import boot, ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params(10, 10)
    p = oracle_params(pr)
    spec = syn.uci_silu_boot_spec(0)
    spec.boot_coeffs = tuple(boot.cos_fit(24, 6, 16))
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    _, evk = H.helrm_model_keygen(ctx, model, 5)
    _, keys = ckks.keygen(p, 5, rot_steps=c.rotation_steps(), h=H_SECRET, conj=True)
    dense, idx = syn.make_queries(spec, 3, seed=8)
    cts, want = [], []
    for q in range(3):
        cd, cs = dlrm.encrypt_query(p, keys, c, dense[q], idx[q], 300 + 2 * q)
        cts.append((import_ct(ctx, cd), import_ct(ctx, cs)))
        want.append(dlrm.infer(p, keys, c, cd, cs))
    srv = H.helrm_server_create(ctx, 1, 4, 0)
    H.helrm_server_add_client(ctx, srv, model, evk)
    outs, _, st = H.helrm_server_run(ctx, srv, np.zeros(3), np.zeros(3, dtype=np.uint32), [x[0] for x in cts],
                                     [x[1] for x in cts])
    assert st["max_batch"] > 1, "the burst should have been batched"
    for q in range(3):
        assert_ct_equal(ctx, outs[q], want[q])


@pytest.mark.parametrize("name,levels", [("criteo_silu_boot_spec", (10, 1)), ("criteo_relu_boot_spec", (12, 1))])
def test_criteo_with_bootstraps_full_size(name, levels):
    """The Criteo-shaped model with polynomial activations at N = 2^16 on the
    bootstrappable chain: SiLU (degree 6) bootstrapped before bottom layer 2
    (256 slots) and on z (512 slots); the ReLU stand-in (degree 14)
    bootstrapped there and before top layer 1 (512 slots).  The library's own
    constants and keys, the client's encryption and the decrypted logit
    against the FP64 model with the same polynomial (3 queries)."""
    from oracle import dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params()
    ctx = gpu_ctx(pr)
    spec = getattr(syn, name)(0)
    w = syn.make_weights(spec, 0)
    model = H.helrm_model_create(ctx, spec, w)
    info = H.helrm_model_info(ctx, model)
    assert (info["lvl_dense"], info["lvl_sel"]) == levels
    sk, evk = H.helrm_model_keygen(ctx, model, 11)
    dense, idx = syn.make_queries(spec, 3, seed=21)
    for q in range(3):
        cd, cs = H.helrm_encrypt_query(ctx, evk, model, dense[q], idx[q], 40 + 2 * q)
        y = H.helrm_infer(ctx, evk, model, cd, cs)
        assert H.helrm_ct_info(ctx, y)[0] == 0
        got = H.helrm_decrypt_logit(ctx, sk, y)[0]
        want = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]
        print(f"{name} query {q}: logit {got:.6f}, FP64 {want:.6f}, error {abs(got - want):.2e}")
        assert abs(got - want) < 1e-2, (q, got, want)
