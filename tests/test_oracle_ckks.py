"""Pins for the oracle's CKKS layer against closed forms, big-integer CRT
checks, an independent ChaCha20 implementation and exact noise bounds."""
import math

import numpy as np
import pytest

from oracle import chacha, ckks, ring


# ---------------------------------------------------------------- ChaCha20
def test_chacha20_quarter_round_rfc8439_2_1_1():
    x = np.zeros((16, 1), dtype=np.uint32)
    x[0], x[1], x[2], x[3] = 0x11111111, 0x01020304, 0x9B8D6F43, 0x01234567
    with np.errstate(over="ignore"):
        chacha._quarter(x, 0, 1, 2, 3)
    assert [int(v[0]) for v in x[:4]] == [0xEA2A92F4, 0xCB1CF8CE, 0x4581472E, 0x5881C4BB]


def test_chacha20_stream_matches_cryptography_library():
    algos = pytest.importorskip("cryptography.hazmat.primitives.ciphers.algorithms")
    ciphers = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    for seed, purpose, index in [(0, 1, 0), (2**64 - 1, 5, (1 << 40) | 3), (1234, 4, 77)]:
        key = seed.to_bytes(8, "little") + bytes(24)
        nonce = purpose.to_bytes(4, "little") + index.to_bytes(8, "little")
        for first_block in [0, 5]:
            # cryptography's ChaCha20 takes 16 bytes: 32-bit counter then the 96-bit nonce
            c = ciphers.Cipher(algos.ChaCha20(key, first_block.to_bytes(4, "little") + nonce), None)
            ks = c.encryptor().update(bytes(64 * 4))
            want = np.frombuffer(ks, dtype="<u4")
            got = chacha.stream_words(seed, purpose, index, 64, first_word=16 * first_block)
            assert np.array_equal(got, want)


def test_samplers_ranges_and_moments():
    t = chacha.ternary(9, chacha.SK, 0, 1 << 16)
    assert set(np.unique(t)) <= {-1, 0, 1}
    frac = [np.mean(t == v) for v in (-1, 0, 1)]
    assert abs(frac[0] - 0.25) < 0.01 and abs(frac[1] - 0.5) < 0.01 and abs(frac[2] - 0.25) < 0.01
    e = chacha.cbd21(9, chacha.PK_E, 0, 1 << 16)
    assert np.max(np.abs(e)) <= 21 and abs(np.var(e) - 10.5) < 0.3 and abs(np.mean(e)) < 0.05
    q = (1 << 40) - 87
    u = chacha.uniform_poly(9, chacha.PK_A, 0, 1 << 14, [q], [0])[0]
    assert np.all(u < q) and abs(np.mean(u.astype(float)) / q - 0.5) < 0.01


# ---------------------------------------------------------------- encoding
def test_encode_n4_by_hand():
    p = ckks.Params(2, [60, 40], 1, 60, 1, 40.0)                # N = 4, n = 2 slots
    z0, z1 = 0.75, -0.5
    r2 = math.sqrt(2.0)
    # sigma^-1 by hand: slots at zeta and zeta^5, zeta = e^(i pi / 4)
    want = [(z0 + z1) / 2, r2 / 4 * (z0 - z1), 0.0, r2 / 4 * (z1 - z0)]
    scale = 2.0**30
    got = ckks.encode_real(p, [z0, z1], scale)
    assert [int(x) for x in got] == [int(np.sign(w) * np.floor(abs(w) * scale + 0.5)) for w in want]
    assert np.allclose(ckks.decode(p, got, scale).real, [z0, z1], atol=2**-28)


def test_encode_fft_equals_direct_definition(small_params):
    p = small_params
    z = np.random.default_rng(0).uniform(-1, 1, p.n)
    a = ckks.encode_real(p, z, p.delta)
    b = ckks.encode_real_direct(p, z, p.delta)
    d = np.abs(a.astype(np.int64) - b.astype(np.int64))
    assert np.max(d) <= 1 and np.sum(d) <= 8         # only FP64 ties may differ
    zd = ckks.decode_direct(p, a, p.delta)
    assert np.allclose(ckks.decode(p, a, p.delta), zd, atol=1e-9)


def test_decode_encode_round_trip(small_params):
    p = small_params
    z = np.random.default_rng(1).uniform(-1, 1, p.n)
    dz = ckks.decode(p, ckks.encode_real(p, z, p.delta), p.delta)
    assert np.max(np.abs(dz.real - z)) < 2**-30 and np.max(np.abs(dz.imag)) < 2**-30


# ---------------------------------------------------------------- encryption
def exact_noise(p, sk, ct, m):
    """e = c0 + c1 s - m as a centred integer (big-integer CRT)."""
    got = ckks.decrypt_poly(p, sk, ct)
    return np.array([int(g) - int(x) for g, x in zip(got, m)], dtype=object)


def test_fresh_encryption_noise_bound(small_params, small_keys):
    p = small_params
    sk, keys = small_keys
    z = np.random.default_rng(2).uniform(-1, 1, p.n)
    m = ckks.encode_real(p, z, p.delta)
    for lvl in [0, 3, p.L]:
        ct = ckks.encrypt(p, keys, m, lvl, p.delta, 77 + lvl)
        e = exact_noise(p, sk, ct, m)
        # |v e_pk + e0 + e1 s|_inf <= 21 N + 21 + 21 N for ternary v, s
        assert max(abs(int(x)) for x in e) <= 42 * p.N + 21
        assert np.max(np.abs(ckks.decrypt(p, sk, ct) - z)) < 1e-6


def test_public_key_relation(small_params, small_keys):
    p = small_params
    sk, keys = small_keys
    mods = p.q_mods(p.L)
    s = ring.from_signed(sk.s, mods)
    e = ring.add(keys.pk_b, ckks.polymul(p, keys.pk_a, s, mods), mods)   # = e_pk
    ec = ckks.crt_centered(p, e, mods)
    assert max(abs(int(x)) for x in ec) <= 21


# ---------------------------------------------------------------- rescale / conversions
def big(p, x, mods):
    """Residues [limbs, N] -> list of integers in [0, prod mods)."""
    M = math.prod(mods)
    out = []
    for c in range(x.shape[1]):
        v = 0
        for l, q in enumerate(mods):
            qh = M // q
            v += int(x[l, c]) * qh * pow(qh % q, -1, q)
        out.append(v % M)
    return out


def test_rescale_is_rounded_division(small_params):
    p = small_params
    lvl = 4
    mods = p.q_mods(lvl)
    rng = np.random.default_rng(3)
    x = np.stack([rng.integers(0, q, 64, dtype=np.uint64) for q in mods])
    x = np.concatenate([x, np.zeros((lvl + 1, p.N - 64), dtype=np.uint64)], axis=1)
    out = ckks.rescale_poly(p, x, lvl)
    X = big(p, x[:, :64], mods)
    Y = big(p, out[:, :64], mods[:-1])
    ql = p.q[lvl]
    Qm = math.prod(mods[:-1])
    for xv, yv in zip(X, Y):
        # round(x / q_l) with ties impossible (q_l odd), as a residue mod Q_{l-1}
        assert yv == ((xv + ql // 2) // ql) % Qm or yv == ((2 * xv + ql) // (2 * ql)) % Qm


def test_fast_base_conversion_overflow_is_bounded(small_params):
    p = small_params
    src = p.q[:3]
    dst = p.q[3:5] + p.p
    rng = np.random.default_rng(4)
    x = np.stack([rng.integers(0, q, 200, dtype=np.uint64) for q in src])
    y = ckks.fast_base_conv(x, src, dst)
    Qs = math.prod(src)
    X = big(p, x, src)
    for c, xv in enumerate(X):
        us = []
        for k, pk in enumerate(dst):
            # y = x + u Qs mod p_k for one integer u with 0 <= u < len(src)
            u = [u for u in range(len(src)) if (xv + u * Qs) % pk == int(y[k, c])]
            assert len(u) == 1
            us.append(u[0])
        assert len(set(us)) == 1


def test_moddown_is_division_by_P_within_K(small_params):
    p = small_params
    lvl = 2
    qp = p.qp_mods(lvl)
    rng = np.random.default_rng(5)
    u = np.zeros((len(qp), p.N), dtype=np.uint64)
    u[:, :100] = np.stack([rng.integers(0, q, 100, dtype=np.uint64) for q in qp])
    out = ckks.moddown(p, u, lvl)
    U = big(p, u[:, :100], qp)
    O = big(p, out[:, :100], p.q_mods(lvl))
    Q = math.prod(p.q_mods(lvl))
    for uv, ov in zip(U, O):
        # out * P = u - ut with ut = u mod P lifted by fast conversion: 0 <= ut < K*P
        lo = (uv - p.K * p.P) // p.P
        hi = uv // p.P
        assert any((v % Q) == ov for v in range(lo, hi + 1))


def test_moddown_rounding_error_has_the_uncorrected_conversions_mean(small_params):
    """Without an overflow correction, ModDown returns floor(u/P) - v with v
    the conversion's overflow (v in [0, K), of mean 1 for K = 3: the floor of
    a sum of three uniforms), so its error against round(u/P) has mean
    -1/2 - 1 = -3/2.  A corrected conversion would give -1/2, an exact
    rounding 0; 1024 random coefficients tell them apart (standard error 0.03)."""
    p = small_params
    lvl = 2
    qp = p.qp_mods(lvl)
    rng = np.random.default_rng(6)
    u = np.stack([rng.integers(0, q, p.N, dtype=np.uint64) for q in qp])
    out = ckks.moddown(p, u, lvl)
    U = big(p, u, qp)
    O = big(p, out, p.q_mods(lvl))
    Q = math.prod(p.q_mods(lvl))
    err = []
    for uv, ov in zip(U, O):
        e = (ov - (2 * uv + p.P) // (2 * p.P)) % Q       # against round(u / P)
        err.append(e - Q if e > Q // 2 else e)
    assert set(err) <= {0, -1, -2, -3}
    assert abs(np.mean(err) + 1.5) < 0.15


# ---------------------------------------------------------------- rotation / key switching
@pytest.mark.parametrize("step", [1, 3, -1, 100, -7])
def test_rotation_is_cyclic_shift(small_params, small_keys, step):
    p = small_params
    sk, keys = small_keys
    z = np.random.default_rng(6).uniform(-1, 1, p.n)
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, z, p.delta), 3, p.delta, 5)
    r = ckks.rotate(p, keys, ct, step)
    assert np.max(np.abs(ckks.decrypt(p, sk, r) - np.roll(z, -step))) < 1e-6


def test_rotation_noise_bound(small_params, small_keys):
    """Key switching adds at most the ModDown rounding plus sum_j |d_j e_j| / P."""
    p = small_params
    sk, keys = small_keys
    z = np.random.default_rng(7).uniform(-1, 1, p.n)
    m = ckks.encode_real(p, z, p.delta)
    lvl = p.L
    ct = ckks.encrypt(p, keys, m, lvl, p.delta, 8)
    r = ckks.rotate(p, keys, ct, 1)
    k = p.galois(1)
    m_rot = ckks.automorphism_signed(p, np.array([int(x) for x in m], dtype=object), k)
    e = exact_noise(p, sk, r, m_rot)
    dnum = p.dnum(lvl)
    qmax = max(p.q)
    fresh = 42 * p.N + 21
    ks = (dnum * p.alpha * qmax * p.N * 21) / p.P + p.K * (p.N + 1)
    assert max(abs(int(x)) for x in e) <= fresh + ks


def test_hoisted_rotation_decrypts_like_plain_rotation(small_params, small_keys):
    """ModUp-then-phi (hoisted) vs phi-then-ModUp: both valid, equal within noise."""
    p = small_params
    sk, keys = small_keys
    z = np.random.default_rng(8).uniform(-1, 1, p.n)
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, z, p.delta), 4, p.delta, 9)
    hoisted = ckks.rotate_hoisted(p, keys, ct, [1, 2, 3])
    k = p.galois(2)
    qm = p.q_mods(4)
    c0, c1 = ckks.automorphism(p, ct.c0, k, qm), ckks.automorphism(p, ct.c1, k, qm)
    u0, u1 = ckks.ks_inner(p, ckks.modup(p, c1, 4), keys.rot[k], 4)
    plain = ckks.Ct(ring.add(c0, ckks.moddown(p, u0, 4), qm), ckks.moddown(p, u1, 4), 4, ct.scale)
    a = ckks.decrypt(p, sk, hoisted[2])
    b = ckks.decrypt(p, sk, plain)
    assert np.max(np.abs(a - b)) < 1e-6 and np.max(np.abs(a - np.roll(z, -2))) < 1e-6


def test_ct_ct_multiply_and_levels(small_params, small_keys):
    p = small_params
    sk, keys = small_keys
    rng = np.random.default_rng(9)
    x, y = rng.uniform(-1, 1, p.n), rng.uniform(-1, 1, p.n)
    a = ckks.encrypt(p, keys, ckks.encode_real(p, x, p.delta), 5, p.delta, 10)
    b = ckks.encrypt(p, keys, ckks.encode_real(p, y, p.delta), 5, p.delta, 11)
    c = ckks.mul(p, keys, a, b)
    assert c.level == 4 and c.scale == p.delta * p.delta / p.q[5]
    assert np.max(np.abs(ckks.decrypt(p, sk, c) - x * y)) < 1e-6
    s = ckks.rescale(p, ckks.mul_pt(p, a, ckks.encode_real(p, y, p.q[5]), p.q[5]))
    assert s.level == 4 and np.max(np.abs(ckks.decrypt(p, sk, s) - x * y)) < 1e-6


def test_sizes_match_paper_orders_of_magnitude():
    """Ciphertext at l = 20 ~ 21 MiB (paper: 10-30 MiB); one eval key with
    dnum = 7 digits over 24 limbs ~ 168 MiB (paper: ~200 MiB)."""
    N, L, K, alpha = 2**16, 20, 3, 3
    ct = 2 * (L + 1) * N * 8
    dnum = -(-(L + 1) // alpha)
    key = dnum * 2 * (L + 1 + K) * N * 8
    assert 10 * 2**20 <= ct <= 30 * 2**20 and round(ct / 2**20) == 21
    assert round(key / 2**20) == 168
