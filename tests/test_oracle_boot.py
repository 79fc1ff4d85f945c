"""Pins of the oracle's bootstrapping (oracle/boot.py) and the pieces it adds
to the scheme (complex encoding, the sparse secret, conjugation), each
against what mathematics fixes: the encoding's definition, brute force,
closed forms, the decrypted integers of every stage, and the message itself
after a whole bootstrap.

The chain is the bootstrappable shape at N = 2^10: q_0 60-bit, 4 x 40-bit
compute primes, 13 x 60-bit primes for the bootstrapping levels, 3 x 60-bit
special primes, a secret with h = 192 non-zero coefficients."""
import math

import numpy as np
import pytest

from oracle import boot, chacha, ckks, poly

LOG_N, N_S, H = 10, 64, 192
Q_BITS = [60] + [40] * 4 + [60] * 13


@pytest.fixture(scope="module")
def setup():
    p = ckks.Params(LOG_N, Q_BITS, 3, 60, 3, 40.0)
    b = boot.prepare(p, boot.BootParams(n_s=N_S))
    sk, keys = ckks.keygen(p, 7, rot_steps=b.rotation_steps(), h=H, conj=True)
    return p, b, sk, keys


@pytest.fixture(scope="module")
def booted(setup):
    p, b, sk, keys = setup
    z = np.random.default_rng(1).uniform(-1, 1, N_S)
    zz = z[np.arange(p.n) % N_S]
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, zz, p.delta), 2, p.delta, 11)
    st = {}
    out = boot.bootstrap(p, keys, b, ct, st)
    return zz, ct, st, out


def test_encode_complex_is_its_definition():
    p = ckks.Params(8, [60, 40], 1, 60, 1, 40.0)
    rng = np.random.default_rng(3)
    z = rng.normal(size=p.n) + 1j * rng.normal(size=p.n)
    m = ckks.encode_complex(p, z, 2.0**30)
    assert np.array_equal(m, ckks.encode_complex_direct(p, z, 2.0**30))
    assert np.max(np.abs(ckks.decode(p, m, 2.0**30) - z)) < 1e-7
    x = rng.normal(size=p.n)
    assert np.array_equal(ckks.encode_complex(p, x, 2.0**30), ckks.encode_real(p, x, 2.0**30))


def test_sparse_secret_brute_force():
    n, h = 512, 37
    s = chacha.sparse_ternary(9, chacha.SK_SPARSE, 0, n, h)
    w = [int(v) for v in chacha.stream_words(9, chacha.SK_SPARSE, 0, 2 * n)]
    chosen = sorted(range(n), key=lambda i: (w[i], i))[:h]
    want = [0] * n
    for i in chosen:
        want[i] = 1 if w[n + i] % 2 == 0 else -1
    assert s.tolist() == want
    assert np.count_nonzero(s) == h
    p = ckks.Params(LOG_N, [60, 40], 1, 60, 1, 40.0)
    assert np.count_nonzero(ckks.secret_key(p, 4, h=H).s) == H
    assert np.count_nonzero(ckks.secret_key(p, 4).s) > p.N // 3      # the dense default (about N/2) is unchanged


def test_conjugation():
    p = ckks.Params(LOG_N, [60, 40, 40], 3, 60, 3, 40.0)
    sk, keys = ckks.keygen(p, 5, relin=False, conj=True)
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, p.n) + 1j * rng.uniform(-1, 1, p.n)
    ct = ckks.encrypt(p, keys, ckks.encode_complex(p, z, p.delta), 2, p.delta, 6)
    out = ckks.conjugate(p, keys, ct)
    got = ckks.decode(p, ckks.decrypt_poly(p, sk, out), out.scale)          # complex slots
    assert np.max(np.abs(got - np.conj(z))) < 1e-6


def test_slot_matrix_closed_forms():
    p = ckks.Params(LOG_N, [60, 40], 1, 60, 1, 40.0)
    U = boot.slot_matrix(N_S)
    # 2 Re(U^H U) = 2 n_s I, so t = (U^H w + U^T conj(w)) / (2 n_s) inverts w = U t for real t
    assert np.max(np.abs(2 * (U.conj().T @ U).real - 2 * N_S * np.eye(2 * N_S))) < 1e-9
    t = np.random.default_rng(5).integers(-1000, 1000, 2 * N_S)
    w = U @ t
    assert np.max(np.abs((U.conj().T @ w + U.T @ np.conj(w)) / (2 * N_S) - t)) < 1e-8
    # the slots of sum_k t_k X^(g k) are U t (period n_s)
    g = p.N // (2 * N_S)
    m = np.zeros(p.N, dtype=np.int64)
    m[::g] = t
    assert np.max(np.abs(ckks.decode(p, m, 1.0) - w[np.arange(p.n) % N_S])) < 1e-6


def test_cos_fit_and_double_angles():
    bp = boot.BootParams(n_s=N_S)
    c = boot.cos_fit(bp.K, bp.r, bp.degree)
    assert all(c[k] == 0.0 for k in range(1, bp.degree + 1, 2)) and c[bp.degree] != 0.0
    Y = (bp.K + 0.5) / 2.0**bp.r
    y = np.linspace(-Y, Y, 100001)
    assert np.max(np.abs(np.polynomial.polynomial.polyval(y, c) - np.cos(2 * np.pi * y))) < 1e-12
    u = np.linspace(-bp.K - 0.01, bp.K + 0.01, 200001)
    v = np.polynomial.polynomial.polyval((u - 0.25) / 2.0**bp.r, c)
    for _ in range(bp.r):
        v = 2 * v * v - 1
    assert np.max(np.abs(v - np.sin(2 * np.pi * u))) < 1e-10
    assert boot.levels_used(bp) == 1 + poly.depth(16) + 6 + 1 == 13


def test_mod_raise_adds_a_small_multiple_of_q0(setup, booted):
    p, b, sk, keys = setup
    zz, ct, st, _ = booted
    low = ckks.decrypt_poly(p, sk, boot.boost(p, ct, b.bp.log2_boost))
    high = ckks.decrypt_poly(p, sk, st["raised"])
    q0 = int(p.q[0])
    diff = [int(hv) - int(lv) for hv, lv in zip(high, low)]
    assert all(d % q0 == 0 for d in diff)
    I = np.array([d // q0 for d in diff])
    assert np.max(np.abs(I)) <= (H + 1) // 2 and np.max(np.abs(I)) >= 1
    assert st["raised"].level == p.L


def test_subsum_is_the_trace(setup, booted):
    p, b, sk, _ = setup
    _, _, st, _ = booted
    g = p.N // (2 * N_S)
    raised = np.array([float(v) for v in ckks.decrypt_poly(p, sk, st["raised"])])
    ss = np.array([float(v) for v in ckks.decrypt_poly(p, sk, st["subsum"])])
    keep = np.arange(p.N) % g == 0
    q0 = float(p.q[0])
    assert np.max(np.abs(ss[keep] - g * raised[keep])) / q0 < 1e-6
    assert np.max(np.abs(ss[~keep])) / q0 < 1e-6


def test_coeff_to_slot_and_eval_mod(setup, booted):
    p, b, sk, _ = setup
    _, _, st, _ = booted
    g = p.N // (2 * N_S)
    u = np.array([float(v) for v in ckks.decrypt_poly(p, sk, st["raised"])])[::g] / float(p.q[0])
    per = np.arange(p.n) % (2 * N_S)
    cts = ckks.decrypt(p, sk, st["cts"]).real
    assert np.max(np.abs(cts - u[per] / 2.0**b.bp.r)) < 1e-10
    em = ckks.decrypt(p, sk, st["evalmod"]).real
    assert np.max(np.abs(em - np.sin(2 * np.pi * u[per]))) < 1e-8


def test_bootstrap_refreshes_the_message(setup, booted):
    p, b, sk, _ = setup
    zz, ct, st, out = booted
    assert out.level == p.L - boot.levels_used(b.bp) == 4
    assert abs(math.log2(out.scale) - 40) < 1e-6
    assert out.scale == boot.out_scale(p, b, ct.scale)                  # the scale is known before the run
    assert st["cts"].scale == boot.scales(p, b)[0] and st["evalmod"].scale == boot.scales(p, b)[1]
    got = ckks.decrypt(p, sk, out)
    assert np.max(np.abs(got.real - zz)) < 1e-6
    assert np.max(np.abs(ckks.decrypt(p, sk, ct).real - zz)) < 1e-6    # the input still decrypts too


def test_bootstrap_on_the_forty_bit_chain_runs_at_lower_precision():
    """The all-40-bit chain of the non-bootstrapped models: CoeffToSlot takes
    two rescales and EvalMod runs at 2^40, so the double angles amplify the
    noise and about 4 bits of a unit message survive (the reason for the
    bootstrappable chain)."""
    p = ckks.Params(LOG_N, [60] + [40] * 20, 3, 60, 3, 40.0)
    b = boot.prepare(p, boot.BootParams(n_s=N_S, cts_levels=2, eval_scale=2.0**40))
    sk, keys = ckks.keygen(p, 7, rot_steps=b.rotation_steps(), h=H, conj=True)
    z = np.random.default_rng(1).uniform(-1, 1, N_S)[np.arange(p.n) % N_S]
    out = boot.bootstrap(p, keys, b, ckks.encrypt(p, keys, ckks.encode_real(p, z, p.delta), 1, p.delta, 3))
    assert out.level == 20 - 14
    err = np.max(np.abs(ckks.decrypt(p, sk, out).real - z))
    assert 1e-4 < err < 0.2


def test_level_plan_segments():
    """Segments between bootstrap points each end at level 0; without points
    the plan is the single as-late-as-possible schedule."""
    from oracle import dlrm
    # Criteo-shaped with SiLU (depth 4): layers cost 5, the last top layer 1, the dot interaction 2
    plan = dlrm.level_plan(4, 3, 4, True, ("b2", "z"))
    assert plan == {"t2": 1, "t1": 6, "t0": 11, "I": 13, "b3": 5, "b2": 10, "b1": 5, "b0": 10, "h": 0}
    plain = dlrm.level_plan(2, 2, 1, True, ())
    lvl_u = (1 + 1) * (2 - 1) + 1
    assert plain["t0"] == lvl_u and plain["I"] == lvl_u + 2 == plain["h"] and plain["b0"] == lvl_u + 2 + 2 * 2
    with pytest.raises(ValueError):
        dlrm.level_plan(2, 2, 1, True, ("b0",))          # before the first layer: not a point


def test_bootstrapped_dlrm_matches_the_cleartext_model():
    """The UCI-shaped SiLU model (concatenation) bootstrapped before bottom
    layer 1 and on z, at N = 2^10 on the bootstrappable chain with 10 compute
    levels: every segment ends at level 0 and the decrypted logit is the
    FP64 model's."""
    from oracle import dlrm
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.boot_params(10, 10)
    p = ckks.Params(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"])
    spec = syn.uci_silu_boot_spec(0)
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    assert (c.lvl_dense, c.lvl_sel, c.lvl_h, c.lvl_z, c.lvl_u) == (5, 1, 0, 6, 6)
    assert {k: (v[0].bp.n_s, v[1]) for k, v in c.boots.items()} == {"b1": (32, 5), "z": (256, 6)}
    assert dlrm.boot_order(c) == ["b1", "z"]
    sk, keys = ckks.keygen(p, 3, rot_steps=c.rotation_steps(), h=H, conj=True)
    dense, idx = syn.make_queries(spec, 1, seed=5)
    cd, cs = dlrm.encrypt_query(p, keys, c, dense[0], idx[0], 100)
    y = dlrm.infer(p, keys, c, cd, cs)
    assert y.level == 0
    got = dlrm.decrypt_logit(p, sk, y)[0]
    want = dlrm.dlrm_cleartext(spec, w, dense[0], idx[0])[0]
    assert abs(got - want) < 1e-4


def test_constant_message_follows_the_sine():
    """With n_s = 1 a constant message z is the constant polynomial
    m = round(Delta z), so EvalMod sees the single value u = 2^b m / q_0 and
    the bootstrap returns sin(2 pi u) / (2 pi u) times z, not z: about
    z (1 - (2 pi u)^2 / 6), 4.6e-6 below 0.9 at 2^b = 2^10 and a 60-bit q_0.
    The output matches the sine to the bootstrap's noise (2e-8), which a
    wrong boost, a dropped 2 pi or a wrong SlotToCoeff constant would miss by
    far more."""
    p = ckks.Params(LOG_N, Q_BITS, 3, 60, 3, 40.0)
    b = boot.prepare(p, boot.BootParams(n_s=1))
    assert len(b.subsum_steps) == LOG_N - 1
    sk, keys = ckks.keygen(p, 7, rot_steps=b.rotation_steps(), h=H, conj=True)
    for z0, seed in ((0.9, 11), (-0.5, 12)):
        ct = ckks.encrypt(p, keys, ckks.encode_real(p, np.full(p.n, z0), p.delta), 2, p.delta, seed)
        got = ckks.decrypt(p, sk, boot.bootstrap(p, keys, b, ct, {})).real
        u = 2.0**b.bp.log2_boost * round(p.delta * z0) / float(p.q[0])
        want = math.sin(2 * math.pi * u) / (2 * math.pi * u) * z0
        assert abs(want - z0) > 5e-7                      # the sine's own departure from z
        assert np.max(np.abs(got - want)) < 1e-7
