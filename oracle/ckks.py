"""RNS-CKKS, written out plainly (test infrastructure only).

Follows the HE-LRM appendix "CKKS operations" (ring R = Z[X]/(X^N+1),
ciphertexts in R_Q^2, Q = prod_{i<=L} q_i; encoding = inverse canonical
embedding, scaled by Delta and rounded; encryption under a public key with
added noise; addition, multiplication, rescaling Q_l -> Q_{l-1}, rotation by
k slots, key switching with a special switching key).  Where the paper is
silent the readings are stated at each function (primes, distributions, key
switching gadget, base conversion, rounding, slot order).

All polynomials here are in the COEFFICIENT domain, numpy uint64 [limbs, N].
Ring products go through the oracle's own textbook NTT (ring.polymul), or the
O(N^2) schoolbook product in the exact cross-checks.  A ciphertext (c0, c1)
at level l decrypts as c0 + c1*s mod Q_l.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import chacha, ring
from .primes import prime_chain, primitive_2n_root


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
class Params:
    """N = 2^log_n; primes q_0..q_L (bit sizes q_bits), K special primes p_k."""

    def __init__(self, log_n: int, q_bits, n_p: int, p_bits: int, alpha: int,
                 log2_scale: float):
        self.log_n = log_n
        self.N = 1 << log_n
        self.n = self.N // 2                    # slots
        self.q, self.p = prime_chain(log_n, list(q_bits), n_p, p_bits)
        self.L = len(self.q) - 1
        self.K = len(self.p)
        self.alpha = alpha
        self.delta = 2.0 ** log2_scale
        self.P = math.prod(self.p)
        two_n = 2 * self.N
        self.psi = {m: primitive_2n_root(m, two_n) for m in self.q + self.p}

    # limb bookkeeping: a QP polynomial at level l holds q_0..q_l then p_0..p_{K-1}
    def q_mods(self, level):
        return self.q[: level + 1]

    def qp_mods(self, level):
        return self.q[: level + 1] + self.p

    def qp_ids(self, level):
        """Positions of the level-l QP limbs in the full QP basis order."""
        return list(range(level + 1)) + list(range(self.L + 1, self.L + 1 + self.K))

    def psis(self, mods):
        return [self.psi[m] for m in mods]

    def dnum(self, level):
        return -(-(level + 1) // self.alpha)

    def digit(self, j, level):
        """Indices of the q-primes in key-switching digit j at level l."""
        return list(range(j * self.alpha, min((j + 1) * self.alpha, level + 1)))

    def galois(self, step: int) -> int:
        """Rotation by `step` slots (left) is X -> X^(5^step mod 2N)."""
        return pow(5, step % self.n, 2 * self.N)

    def conj_galois(self) -> int:
        """Complex conjugation of every slot is X -> X^(2N-1) = X^(-1)."""
        return 2 * self.N - 1


# EXACT = True: every ring product is the O(N^2) schoolbook negacyclic
# convolution (the product's definition, X^N = -1) instead of the textbook NTT;
# both are exact, so every result is the same, only slower (the "oracle-exact"
# timing of the tiny lookup).  Limbs run on a thread pool (the C core releases
# the GIL), which changes no result.
EXACT = False


def _schoolbook_limbs(a, b, mods):
    from concurrent.futures import ThreadPoolExecutor
    a2, b2 = np.atleast_2d(a), np.atleast_2d(b)
    with ThreadPoolExecutor(max_workers=max(1, min(len(mods), os.cpu_count() or 1))) as ex:
        rows = list(ex.map(lambda i: ring.schoolbook(a2[i], b2[i], int(mods[i])), range(len(mods))))
    return np.stack(rows)


def polymul(p: Params, a, b, mods):
    if EXACT:
        return _schoolbook_limbs(a, b, mods)
    return ring.polymul(a, b, mods, p.psis(mods))


# --------------------------------------------------------------------------
# Encoding (appendix: inverse FFT, scale by Delta, round)
# --------------------------------------------------------------------------
def _slot_exponents(p: Params) -> np.ndarray:
    """5^j mod 2N for j < n: slot j is the evaluation at zeta^(5^j), zeta = e^(i pi/N)."""
    e = np.empty(p.n, dtype=np.int64)
    x = 1
    for j in range(p.n):
        e[j] = x
        x = x * 5 % (2 * p.N)
    return e


def round_half_away(x: np.ndarray):
    r = np.sign(x) * np.floor(np.abs(x) + 0.5)
    if np.max(np.abs(r), initial=0.0) < 2.0**62:
        return r.astype(np.int64)
    return np.array([int(v) for v in r], dtype=object)


def encode_real(p: Params, z, scale: float) -> np.ndarray:
    """m = round(scale * sigma^-1(z)) for real slots z (zero-padded to n).

    sigma^-1(z)_k = (1/N) sum_j (z_j zeta^(-5^j k) + conj(z_j) zeta^(5^j k)),
    evaluated with one length-2N FFT of the vector that holds z_j at 5^j and
    conj(z_j) at -5^j (mod 2N).
    """
    v = np.zeros(p.n, dtype=np.complex128)
    z = np.asarray(z, dtype=np.float64)
    v[: z.shape[0]] = z
    e = _slot_exponents(p)
    w = np.zeros(2 * p.N, dtype=np.complex128)
    w[e] = v
    w[(2 * p.N - e) % (2 * p.N)] = np.conj(v)
    m = np.fft.fft(w)[: p.N].real / p.N
    return round_half_away(scale * m)


def encode_complex(p: Params, z, scale: float) -> np.ndarray:
    """encode_real for complex slots: the same length-2N FFT of the vector
    that holds z_j at 5^j and conj(z_j) at -5^j (mod 2N), whose real part is
    sigma^-1(z) scaled by N."""
    v = np.zeros(p.n, dtype=np.complex128)
    z = np.asarray(z, dtype=np.complex128)
    v[: z.shape[0]] = z
    e = _slot_exponents(p)
    w = np.zeros(2 * p.N, dtype=np.complex128)
    w[e] = v
    w[(2 * p.N - e) % (2 * p.N)] = np.conj(v)
    m = np.fft.fft(w)[: p.N].real / p.N
    return round_half_away(scale * m)


def encode_complex_direct(p: Params, z, scale: float) -> np.ndarray:
    """m_k = round(scale (1/N) sum_j 2 Re(z_j zeta^(-5^j k))), the definition (small N only)."""
    zz = np.zeros(p.n, dtype=np.complex128)
    z = np.asarray(z, dtype=np.complex128)
    zz[: z.shape[0]] = z
    e = _slot_exponents(p)
    ang = np.pi * np.outer(e, np.arange(p.N)) / p.N
    m = 2.0 * np.real(zz[:, None] * np.exp(-1j * ang)).sum(axis=0) / p.N
    return round_half_away(scale * m)


def encode_real_direct(p: Params, z, scale: float) -> np.ndarray:
    """The same map as a direct O(N n) sum (small N only)."""
    z = np.asarray(z, dtype=np.float64)
    zz = np.zeros(p.n, dtype=np.complex128)
    zz[: z.shape[0]] = z
    e = _slot_exponents(p)
    k = np.arange(p.N)
    ang = np.pi * np.outer(e, k) / p.N                    # [n, N]
    m = 2.0 * np.real(zz[:, None] * np.exp(-1j * ang)).sum(axis=0) / p.N
    return round_half_away(scale * m)


def decode(p: Params, m, scale: float, n_slots: int | None = None) -> np.ndarray:
    """z_j = m(zeta^(5^j)) / scale for centred integer coefficients m."""
    v = np.zeros(2 * p.N, dtype=np.complex128)
    v[: p.N] = np.array([float(x) for x in m]) if np.asarray(m).dtype == object else np.asarray(m, dtype=np.float64)
    g = np.fft.ifft(v) * (2 * p.N)                       # g[t] = sum_k v_k e^(2 pi i t k / 2N)
    z = g[_slot_exponents(p)] / scale
    return z[: (n_slots or p.n)]


def decode_direct(p: Params, m, scale: float) -> np.ndarray:
    mf = np.asarray([float(x) for x in m])
    e = _slot_exponents(p)
    ang = np.pi * np.outer(e, np.arange(p.N)) / p.N
    return (mf[None, :] * np.exp(1j * ang)).sum(axis=1) / scale


# --------------------------------------------------------------------------
# Ring helpers
# --------------------------------------------------------------------------
def automorphism(p: Params, a: np.ndarray, k: int, mods) -> np.ndarray:
    """phi_k(a)(X) = a(X^k): coefficient i moves to i*k mod 2N, negated past N."""
    a = np.atleast_2d(a)
    idx = (np.arange(p.N, dtype=np.int64) * k) % (2 * p.N)
    dest = idx % p.N
    flip = idx >= p.N
    out = np.empty_like(a)
    for l, q in enumerate(mods):
        q = np.uint64(q)
        out[l, dest] = np.where(flip, (q - a[l]) % q, a[l])
    return out


def automorphism_signed(p: Params, s: np.ndarray, k: int) -> np.ndarray:
    idx = (np.arange(p.N, dtype=np.int64) * k) % (2 * p.N)
    out = np.empty_like(s)
    out[idx % p.N] = np.where(idx >= p.N, -s, s)
    return out


def lift_times_P(p: Params, a: np.ndarray, level: int) -> np.ndarray:
    """The Q-level polynomial a viewed in QP and multiplied by P (0 on the P limbs)."""
    mods = p.q_mods(level)
    top = ring.mul_scalar(a, [p.P % q for q in mods], mods)
    return np.concatenate([top, np.zeros((p.K, p.N), dtype=np.uint64)])


# --------------------------------------------------------------------------
# Keys
# --------------------------------------------------------------------------
@dataclass
class SecretKey:
    s: np.ndarray                                 # signed ternary coefficients


@dataclass
class SwitchKey:
    """Digits j: (b_j, a_j) over the full QP basis at the top level."""
    b: list
    a: list


@dataclass
class Keys:
    seed: int
    pk_b: np.ndarray
    pk_a: np.ndarray
    relin: SwitchKey | None = None
    rot: dict = field(default_factory=dict)       # galois element -> SwitchKey


def secret_key(p: Params, seed: int, h: int = 0) -> SecretKey:
    """Dense ternary CBD(1) secret (h = 0), or exactly h coefficients in
    {-1, +1} (h > 0): the sparse secret a bootstrapping key set needs, so
    that the multiple of q_0 that ModRaise adds stays small (|I| <= (h+1)/2)."""
    if h:
        return SecretKey(chacha.sparse_ternary(seed, chacha.SK_SPARSE, 0, p.N, h))
    return SecretKey(chacha.ternary(seed, chacha.SK, 0, p.N))


def public_key(p: Params, seed: int, sk: SecretKey):
    """pk = (b, a) = (-a s + e, a) over q_0..q_L."""
    mods = p.q_mods(p.L)
    a = chacha.uniform_poly(seed, chacha.PK_A, 0, p.N, mods, list(range(p.L + 1)))
    e = ring.from_signed(chacha.cbd21(seed, chacha.PK_E, 0, p.N), mods)
    s = ring.from_signed(sk.s, mods)
    b = ring.add(ring.neg(polymul(p, a, s, mods), mods), e, mods)
    return b, a


def switch_key(p: Params, seed: int, sk: SecretKey, s_prime_mod: np.ndarray, key_id: int) -> SwitchKey:
    """Hybrid key-switching key from s' to s (the reading of the paper's
    "special switching key").

    Digit j covers primes D_j = [j*alpha, (j+1)*alpha) of q_0..q_L.  Over every
    limb of QP:  b_j = -a_j s + e_j + [P]_{q_i} s'  if q_i is in D_j, else
    b_j = -a_j s + e_j.  (The gadget value P * Qtilde_j is P mod q_i on D_j and
    0 on every other limb.)  `s_prime_mod` holds s' reduced mod each limb of
    the top-level QP basis.
    """
    mods = p.qp_mods(p.L)
    ids = p.qp_ids(p.L)
    s = ring.from_signed(sk.s, mods)
    bs, as_ = [], []
    for j in range(p.dnum(p.L)):
        index = (key_id << 8) | j
        a = chacha.uniform_poly(seed, chacha.KSK_A, index, p.N, mods, ids)
        e = ring.from_signed(chacha.cbd21(seed, chacha.KSK_E, index, p.N), mods)
        b = ring.add(ring.neg(polymul(p, a, s, mods), mods), e, mods)
        for i in p.digit(j, p.L):
            gad = ring.mul_scalar(s_prime_mod[i:i + 1], [p.P % p.q[i]], [p.q[i]])
            b[i] = ring.add(b[i], gad, [p.q[i]])[0]
        bs.append(b)
        as_.append(a)
    return SwitchKey(bs, as_)


def keygen(p: Params, seed: int, rot_steps=(), relin: bool = True, h: int = 0, conj: bool = False):
    """Secret, public, relinearisation and rotation keys; with conj the key of
    the conjugation X -> X^(2N-1) as well (its key id is that element)."""
    sk = secret_key(p, seed, h)
    pk_b, pk_a = public_key(p, seed, sk)
    keys = Keys(seed, pk_b, pk_a)
    mods = p.qp_mods(p.L)
    s_mod = ring.from_signed(sk.s, mods)
    if relin:
        s2 = polymul(p, s_mod, s_mod, mods)
        keys.relin = switch_key(p, seed, sk, s2, 0)
    for st in sorted(set(int(r) % p.n for r in rot_steps) - {0}):
        k = p.galois(st)
        if k in keys.rot:
            continue
        sk_rot = ring.from_signed(automorphism_signed(p, sk.s, k), mods)
        keys.rot[k] = switch_key(p, seed, sk, sk_rot, k)
    if conj:
        k = p.conj_galois()
        keys.rot[k] = switch_key(p, seed, sk, ring.from_signed(automorphism_signed(p, sk.s, k), mods), k)
    return sk, keys


# --------------------------------------------------------------------------
# Ciphertexts
# --------------------------------------------------------------------------
@dataclass
class Ct:
    c0: np.ndarray
    c1: np.ndarray
    level: int
    scale: float


def encrypt(p: Params, keys: Keys, m, level: int, scale: float, seed: int) -> Ct:
    """(v*b + e0 + m, v*a + e1) with v ternary, e0, e1 CBD(21) (reading of 'some noise')."""
    mods = p.q_mods(level)
    v = ring.from_signed(chacha.ternary(seed, chacha.ENC_V, 0, p.N), mods)
    e0 = ring.from_signed(chacha.cbd21(seed, chacha.ENC_E0, 0, p.N), mods)
    e1 = ring.from_signed(chacha.cbd21(seed, chacha.ENC_E1, 0, p.N), mods)
    mm = ring.from_signed(m, mods)
    c0 = ring.add(ring.add(polymul(p, v, keys.pk_b[: level + 1], mods), e0, mods), mm, mods)
    c1 = ring.add(polymul(p, v, keys.pk_a[: level + 1], mods), e1, mods)
    return Ct(c0, c1, level, scale)


def crt_centered(p: Params, x: np.ndarray, mods) -> np.ndarray:
    """Centred integer representative in (-Q/2, Q/2] of residues x (object array)."""
    Q = math.prod(mods)
    acc = np.zeros(x.shape[1], dtype=object)
    for l, q in enumerate(mods):
        qh = Q // q
        c = qh * pow(qh % q, -1, q)
        acc = acc + x[l].astype(object) * c
    acc = acc % Q
    return np.where(acc > Q // 2, acc - Q, acc)


def decrypt_poly(p: Params, sk: SecretKey, ct: Ct) -> np.ndarray:
    """m = c0 + c1*s mod Q_l, centred (full CRT, no shortcut)."""
    mods = p.q_mods(ct.level)
    s = ring.from_signed(sk.s, mods)
    m = ring.add(ct.c0, polymul(p, ct.c1, s, mods), mods)
    return crt_centered(p, m, mods)


def decrypt(p: Params, sk: SecretKey, ct: Ct, n_slots=None) -> np.ndarray:
    return decode(p, decrypt_poly(p, sk, ct), ct.scale, n_slots).real


def _check_same(a: Ct, b: Ct):
    if a.level != b.level:
        raise ValueError("level mismatch")
    if abs(a.scale - b.scale) > 1e-9 * a.scale:
        raise ValueError("scale mismatch")


def add(p: Params, a: Ct, b: Ct) -> Ct:
    _check_same(a, b)
    mods = p.q_mods(a.level)
    return Ct(ring.add(a.c0, b.c0, mods), ring.add(a.c1, b.c1, mods), a.level, a.scale)


def sub(p: Params, a: Ct, b: Ct) -> Ct:
    _check_same(a, b)
    mods = p.q_mods(a.level)
    return Ct(ring.sub(a.c0, b.c0, mods), ring.sub(a.c1, b.c1, mods), a.level, a.scale)


def add_pt(p: Params, a: Ct, m, pt_scale: float) -> Ct:
    if abs(a.scale - pt_scale) > 1e-9 * a.scale:
        raise ValueError("scale mismatch")
    mods = p.q_mods(a.level)
    return Ct(ring.add(a.c0, ring.from_signed(m, mods), mods), a.c1.copy(), a.level, a.scale)


def mul_pt(p: Params, a: Ct, m, pt_scale: float) -> Ct:
    mods = p.q_mods(a.level)
    mm = ring.from_signed(m, mods)
    return Ct(polymul(p, a.c0, mm, mods), polymul(p, a.c1, mm, mods), a.level, a.scale * pt_scale)


def drop_level(p: Params, a: Ct, level: int) -> Ct:
    if level > a.level:
        raise ValueError("cannot raise a level")
    return Ct(a.c0[: level + 1].copy(), a.c1[: level + 1].copy(), level, a.scale)


def rescale_poly(p: Params, x: np.ndarray, level: int) -> np.ndarray:
    """Drop q_l: out_i = (x_i - r) * q_l^-1 mod q_i, with r = [x]_{q_l} centred
    in (-q_l/2, q_l/2].  This is round(x / q_l) exactly."""
    ql = p.q[level]
    r = x[level].astype(object)
    r = np.where(r > ql // 2, r - ql, r)
    mods = p.q_mods(level - 1)
    rr = ring.from_signed(r, mods)
    d = ring.sub(x[:level], rr, mods)
    return ring.mul_scalar(d, [pow(ql, -1, q) for q in mods], mods)


def rescale(p: Params, a: Ct) -> Ct:
    if a.level < 1:
        raise ValueError("no level left to rescale")
    return Ct(rescale_poly(p, a.c0, a.level), rescale_poly(p, a.c1, a.level),
              a.level - 1, a.scale / p.q[a.level])


# --------------------------------------------------------------------------
# Basis conversion, ModUp, ModDown, key switching
# --------------------------------------------------------------------------
def fast_base_conv(x: np.ndarray, src, dst) -> np.ndarray:
    """y_k = sum_i [x_i * (Qs/q_i)^-1]_{q_i} * (Qs/q_i mod p_k)  mod p_k.

    No correction of the overflow: the result is x + u*Qs mod p_k for some
    integer 0 <= u < len(src) (the reading used for ModUp and ModDown).
    """
    Qs = math.prod(src)
    N = x.shape[1]
    y = np.zeros((len(dst), N), dtype=np.uint64)
    for i, qi in enumerate(src):
        qh = Qs // qi
        t = ring.mul_scalar(x[i:i + 1], [pow(qh % qi, -1, qi)], [qi])[0]
        for k, pk in enumerate(dst):
            y[k] = ring.add(y[k:k + 1], ring.mul_scalar(t[None, :], [qh % pk], [pk]), [pk])[0]
    return y


def modup(p: Params, c: np.ndarray, level: int) -> list:
    """Decompose c (level l, coefficient form) into dnum_l digits, each
    extended to all level-l QP limbs: digit j keeps its own residues and
    base-converts them to the other q-limbs and to the P-limbs."""
    qp = p.qp_mods(level)
    out = []
    for j in range(p.dnum(level)):
        dig = p.digit(j, level)
        src = [p.q[i] for i in dig]
        others = [i for i in range(len(qp)) if i not in dig]
        conv = fast_base_conv(c[dig], src, [qp[i] for i in others])
        d = np.empty((len(qp), p.N), dtype=np.uint64)
        d[dig] = c[dig]
        d[others] = conv
        out.append(d)
    return out


def moddown(p: Params, u: np.ndarray, level: int) -> np.ndarray:
    """QP -> Q: out_i = (u_i - FBC_{P->Q}([u]_P)_i) * P^-1 mod q_i (no P/2 offset)."""
    mods = p.q_mods(level)
    y = fast_base_conv(u[level + 1:], p.p, mods)
    d = ring.sub(u[: level + 1], y, mods)
    return ring.mul_scalar(d, [pow(p.P % q, -1, q) for q in mods], mods)


def ks_inner(p: Params, digits: list, key: SwitchKey, level: int):
    """(u0, u1) = sum_j d_j * (b_j, a_j) over the level-l QP limbs."""
    mods = p.qp_mods(level)
    ids = p.qp_ids(level)
    u0 = np.zeros((len(mods), p.N), dtype=np.uint64)
    u1 = np.zeros_like(u0)
    for j, d in enumerate(digits):
        u0 = ring.add(u0, polymul(p, d, key.b[j][ids], mods), mods)
        u1 = ring.add(u1, polymul(p, d, key.a[j][ids], mods), mods)
    return u0, u1


def _key_for(keys: Keys, k: int) -> SwitchKey:
    if k not in keys.rot:
        raise KeyError(f"no rotation key for galois element {k}")
    return keys.rot[k]


def rotate_hoisted(p: Params, keys: Keys, a: Ct, steps) -> dict:
    """Rotations sharing one ModUp of c1: for each step, phi is applied to the
    extended digits, then the key inner product, then ModDown, plus phi(c0)."""
    digits = modup(p, a.c1, a.level)
    qp = p.qp_mods(a.level)
    mods = p.q_mods(a.level)
    out = {}
    for st in steps:
        if st % p.n == 0:
            out[st] = Ct(a.c0.copy(), a.c1.copy(), a.level, a.scale)
            continue
        k = p.galois(st)
        dr = [automorphism(p, d, k, qp) for d in digits]
        u0, u1 = ks_inner(p, dr, _key_for(keys, k), a.level)
        c0 = ring.add(automorphism(p, a.c0, k, mods), moddown(p, u0, a.level), mods)
        out[st] = Ct(c0, moddown(p, u1, a.level), a.level, a.scale)
    return out


def rotate(p: Params, keys: Keys, a: Ct, step: int) -> Ct:
    return rotate_hoisted(p, keys, a, [step])[step]


def apply_galois(p: Params, keys: Keys, a: Ct, k: int) -> Ct:
    """X -> X^k with the key switch from phi_k(s) back to s, in the order of
    a hoisted rotation: ModUp of c1, phi_k on the extended digits, the key
    inner product, ModDown, plus phi_k(c0).  (ModUp and phi_k do not commute
    word for word: the base conversion of a negated residue differs.)"""
    digits = modup(p, a.c1, a.level)
    qp = p.qp_mods(a.level)
    mods = p.q_mods(a.level)
    u0, u1 = ks_inner(p, [automorphism(p, d, k, qp) for d in digits], _key_for(keys, k), a.level)
    c0 = ring.add(automorphism(p, a.c0, k, mods), moddown(p, u0, a.level), mods)
    return Ct(c0, moddown(p, u1, a.level), a.level, a.scale)


def conjugate(p: Params, keys: Keys, a: Ct) -> Ct:
    """Every slot z_j -> conj(z_j)."""
    return apply_galois(p, keys, a, p.conj_galois())


def tensor(p: Params, a: Ct, b: Ct):
    if a.level != b.level:
        raise ValueError("level mismatch")
    mods = p.q_mods(a.level)
    d0 = polymul(p, a.c0, b.c0, mods)
    d1 = ring.add(polymul(p, a.c0, b.c1, mods), polymul(p, a.c1, b.c0, mods), mods)
    d2 = polymul(p, a.c1, b.c1, mods)
    return d0, d1, d2


def relinearize(p: Params, keys: Keys, d, level: int, scale: float) -> Ct:
    d0, d1, d2 = d
    mods = p.q_mods(level)
    u0, u1 = ks_inner(p, modup(p, d2, level), keys.relin, level)
    return Ct(ring.add(d0, moddown(p, u0, level), mods),
              ring.add(d1, moddown(p, u1, level), mods), level, scale)


def mul(p: Params, keys: Keys, a: Ct, b: Ct) -> Ct:
    """ct x ct: tensor, relinearize with the s^2 key, rescale."""
    d = tensor(p, a, b)
    return rescale(p, relinearize(p, keys, d, a.level, a.scale * b.scale))


def square(p: Params, keys: Keys, a: Ct) -> Ct:
    return mul(p, keys, a, a)
