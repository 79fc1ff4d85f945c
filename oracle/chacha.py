"""ChaCha20 keystream and the CKKS samplers built on it (test infrastructure).

The paper only says that encryption adds "some random noise" (appendix
"CKKS operations").  To make ciphertexts reproducible bit for bit, both sides
derive every random value from the ChaCha20 block function of RFC 8439,
each written independently from that definition:

  key    = the 64-bit seed, little-endian, followed by 24 zero bytes;
  nonce  = three 32-bit words (purpose, index low, index high);
  block c of a stream = ChaCha20(key, counter=c, nonce), 16 words;
  the stream is blocks 0, 1, 2, ... concatenated (word w = block w//16,
  word w%16).

Samplers (the reading of the paper's unspecified distributions):
  uniform mod q : coefficient t of a polynomial over several limbs
                  (t = limb * N + i, the limb counted in the full QP basis
                  order) takes words 4t..4t+3 as (lo, hi) 64-bit halves and
                  returns (hi * 2^64 + lo) mod q.
  ternary CBD(1): coefficient i takes word i: (w & 1) - ((w >> 1) & 1).
  CBD(21)       : coefficient i takes words 2i, 2i+1 as x = w0 | w1 << 32 and
                  returns popcount(x & M) - popcount((x >> 21) & M),
                  M = 2^21 - 1 (standard deviation sqrt(10.5) ~ 3.24, |e| <= 21).
  sparse ternary: exactly h non-zero coefficients (the secret of the
                  bootstrapping key set).  Word i is the priority of
                  coefficient i; the h coefficients with the smallest
                  (priority, i) pairs are non-zero, and coefficient i is
                  +1 if bit 0 of word n + i is 0, else -1.
"""
from __future__ import annotations

import numpy as np

from . import ring

# Stream purposes (nonce word 0).
SK, PK_A, PK_E, KSK_A, KSK_E, ENC_V, ENC_E0, ENC_E1 = 1, 2, 3, 4, 5, 6, 7, 8
SK_SPARSE = 9

_CONST = (0x61707865, 0x3320646E, 0x79622D32, 0x6B206574)   # "expand 32-byte k"


def _rotl(x: np.ndarray, r: int) -> np.ndarray:
    return (x << np.uint32(r)) | (x >> np.uint32(32 - r))


def _quarter(x, a, b, c, d):
    x[a] += x[b]; x[d] ^= x[a]; x[d] = _rotl(x[d], 16)
    x[c] += x[d]; x[b] ^= x[c]; x[b] = _rotl(x[b], 12)
    x[a] += x[b]; x[d] ^= x[a]; x[d] = _rotl(x[d], 8)
    x[c] += x[d]; x[b] ^= x[c]; x[b] = _rotl(x[b], 7)


def chacha20_blocks(key_words, nonce_words, counters) -> np.ndarray:
    """RFC 8439 Sec. 2.3 block function for many counters: returns [n, 16] uint32."""
    counters = np.asarray(counters, dtype=np.uint32)
    n = counters.shape[0]
    st = np.empty((16, n), dtype=np.uint32)
    for i in range(4):
        st[i] = _CONST[i]
    for i in range(8):
        st[4 + i] = np.uint32(key_words[i])
    st[12] = counters
    for i in range(3):
        st[13 + i] = np.uint32(nonce_words[i])
    x = st.copy()
    with np.errstate(over="ignore"):
        for _ in range(10):                      # 20 rounds = 10 double rounds
            _quarter(x, 0, 4, 8, 12)
            _quarter(x, 1, 5, 9, 13)
            _quarter(x, 2, 6, 10, 14)
            _quarter(x, 3, 7, 11, 15)
            _quarter(x, 0, 5, 10, 15)
            _quarter(x, 1, 6, 11, 12)
            _quarter(x, 2, 7, 8, 13)
            _quarter(x, 3, 4, 9, 14)
        x += st
    return x.T.copy()


def stream_words(seed: int, purpose: int, index: int, n_words: int,
                 first_word: int = 0) -> np.ndarray:
    """Words [first_word, first_word + n_words) of the stream (seed, purpose, index)."""
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF, 0, 0, 0, 0, 0, 0]
    nonce = [purpose & 0xFFFFFFFF, index & 0xFFFFFFFF, (index >> 32) & 0xFFFFFFFF]
    b0 = first_word // 16
    b1 = (first_word + n_words + 15) // 16
    blocks = chacha20_blocks(key, nonce, np.arange(b0, b1, dtype=np.uint64).astype(np.uint32))
    flat = blocks.reshape(-1)
    off = first_word - 16 * b0
    return flat[off:off + n_words]


def uniform_poly(seed: int, purpose: int, index: int, n: int, moduli,
                 limb_ids) -> np.ndarray:
    """Uniform residues for the limbs `limb_ids` (positions in the QP order)."""
    rows = []
    for lid, q in zip(limb_ids, moduli):
        w = stream_words(seed, purpose, index, 4 * n, first_word=4 * n * lid).astype(np.uint64)
        w = w.reshape(n, 4)
        lo = w[:, 0] | (w[:, 1] << np.uint64(32))
        hi = w[:, 2] | (w[:, 3] << np.uint64(32))
        rows.append(ring.reduce128(hi, lo, [q])[0])
    return np.ascontiguousarray(np.stack(rows))


def ternary(seed: int, purpose: int, index: int, n: int) -> np.ndarray:
    w = stream_words(seed, purpose, index, n).astype(np.int64)
    return (w & 1) - ((w >> 1) & 1)


def _popcount64(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64)
    c = np.zeros(x.shape, dtype=np.int64)
    for _ in range(64):
        c += (x & np.uint64(1)).astype(np.int64)
        x >>= np.uint64(1)
    return c


def cbd21(seed: int, purpose: int, index: int, n: int) -> np.ndarray:
    w = stream_words(seed, purpose, index, 2 * n).astype(np.uint64).reshape(n, 2)
    x = w[:, 0] | (w[:, 1] << np.uint64(32))
    m = np.uint64((1 << 21) - 1)
    return _popcount64(x & m) - _popcount64((x >> np.uint64(21)) & m)


def sparse_ternary(seed: int, purpose: int, index: int, n: int, h: int) -> np.ndarray:
    """h coefficients in {-1, +1} at the h smallest (priority, position) pairs, the rest 0."""
    if not 0 < h <= n:
        raise ValueError("need 0 < h <= n")
    w = stream_words(seed, purpose, index, 2 * n).astype(np.int64)
    order = np.lexsort((np.arange(n), w[:n]))          # by priority, then by position
    s = np.zeros(n, dtype=np.int64)
    pos = order[:h]
    s[pos] = 1 - 2 * (w[n + pos] & 1)
    return s
