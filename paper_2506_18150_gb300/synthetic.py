"""Seeded synthetic workloads shaped like the HE-LRM experiments.

The UCI Heart Disease and Criteo datasets and trained DLRM weights are not
available, so every input is drawn here from a fixed seed with the shapes of
the paper's workloads (Sec. 5.1, Sec. 5.4): dense features, embedding-table
cardinalities, compressed tables, MLP weights and query indices.  FHE cost is
data-oblivious, so only the shapes matter for time; the values matter for
correctness checks only.

This module holds no homomorphic arithmetic and imports nothing from the
library or from the oracle; both the library's tests/bench and the oracle
consume what it returns.  The one computation in it is the weight
calibration: a plain FP64 forward pass used only to rescale each layer so its
pre-activations have unit RMS over 256 seeded calibration queries (the x^2
activation would otherwise overflow the CKKS message range).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# CKKS parameter presets (bit sizes; the primes are derived by each side)
# --------------------------------------------------------------------------
PARAMS = {
    # N = 2^13, three 50-bit primes + one 50-bit special prime, one prime per digit
    "tiny": dict(log_n=13, q_bits=[50, 50, 50], n_p=1, p_bits=50, alpha=1, log2_scale=40.0),
    # N = 2^16, 60-bit base prime + 20 x 40-bit, three 60-bit special primes
    "full": dict(log_n=16, q_bits=[60] + [40] * 20, n_p=3, p_bits=60, alpha=3, log2_scale=40.0),
}


def boot_params(log_n: int = 16, n_compute: int = 13) -> dict:
    """The bootstrappable chain: q_0 60-bit, n_compute x 40-bit primes for the
    model's levels, 13 x 60-bit primes for bootstrapping (CoeffToSlot 1,
    the degree-16 cosine 5, 6 double angles, SlotToCoeff 1), 3 x 60-bit
    special primes; at N = 2^16 with 13 compute primes log2(QP) = 1540."""
    return dict(log_n=log_n, q_bits=[60] + [40] * n_compute + [60] * 13, n_p=3, p_bits=60, alpha=3,
                log2_scale=40.0)


def reduced_params(log_n: int, n_levels: int) -> dict:
    """The 'full' chain shape at a smaller ring degree and depth (tests)."""
    return dict(log_n=log_n, q_bits=[60] + [40] * n_levels, n_p=3, p_bits=60, alpha=3,
                log2_scale=40.0)


# --------------------------------------------------------------------------
# Model shapes
# --------------------------------------------------------------------------
@dataclass
class DLRMSpec:
    name: str
    n_dense: int
    bottom: list            # layer widths, [n_dense, ..., dim]
    top: list               # layer widths, [top_in, ..., 1]
    cards: list             # rows k_t of each embedding table
    base: int               # digit base p
    dim: int = 16
    interaction: str = "dot"    # "dot" (pairwise) or "concat" (the paper's choice)
    threshold: int | None = None    # tables with more rows are digit-decomposed (None: base)
    act: tuple | None = None    # activation polynomial a_0..a_d (power basis); None: x^2
    boot: tuple = ()            # bootstrap points: "b<i>" before bottom layer i, "z" on z, "t<i>" before top layer i
    boot_coeffs: tuple | None = None    # the bootstraps' cosine polynomial (None: each side's own fit)


def act_apply(spec: DLRMSpec, v):
    """The model's activation on cleartext values: x^2, or its polynomial."""
    if spec.act is None:
        return v ** 2
    return np.polynomial.polynomial.polyval(v, np.asarray(spec.act, dtype=np.float64))


def _lsq_fit(f, degree: int, bound: float) -> tuple:
    # least squares at 1024 Chebyshev points of [-bound, bound], in the
    # Chebyshev basis of the scaled interval, then converted to powers of x
    t = np.cos(np.pi * (np.arange(1024) + 0.5) / 1024)
    cheb = np.polynomial.chebyshev.chebfit(t, f(bound * t), degree)
    pw = np.polynomial.chebyshev.cheb2poly(cheb)
    a = [float(pw[k] / bound ** k) for k in range(degree + 1)]
    # terms that vanish by symmetry come out at rounding level: make them exact
    # zeros (the evaluation then skips their powers), and drop trailing zeros
    top = max(abs(v) for v in a)
    a = [0.0 if abs(v) < 1e-12 * top else v for v in a]
    while len(a) > 1 and a[-1] == 0.0:
        a.pop()
    return tuple(a)


def silu_poly(degree: int = 7, bound: float = 6.0) -> tuple:
    """Power-basis coefficients of a least-squares fit of SiLU(x) = x / (1 +
    e^-x) on [-bound, bound] (the paper's SiLU activation, Sec. 5.4; its
    coefficients are not printed, so this fit stands in for them)."""
    return _lsq_fit(lambda x: x / (1.0 + np.exp(-x)), degree, bound)


def relu_poly(degree: int = 8, bound: float = 6.0) -> tuple:
    """Power-basis coefficients of a least-squares fit of max(x, 0) on
    [-bound, bound] (a single low-degree stand-in for the paper's composite
    ReLU polynomials, which need bootstrapping depth)."""
    return _lsq_fit(lambda x: np.maximum(x, 0.0), degree, bound)


def n_digits(k: int, p: int) -> int:
    """Number of compressed tables for k rows in base p (k <= p keeps one plain table)."""
    if k <= p:
        return 1
    ell, cap = 1, p
    while cap < k:
        cap *= p
        ell += 1
    return ell


def table_rows(k: int, p: int, threshold=None) -> list:
    """Rows of the tables that replace one of k rows: itself if it is not
    compressed (k <= threshold, which defaults to p), else l digit tables of p rows."""
    return [k] if k <= (p if threshold is None else threshold) else [p] * n_digits(k, p)


def top_input_width(spec: DLRMSpec) -> int:
    b = len(spec.cards) + 1
    if spec.interaction == "dot":
        return spec.dim + b * (b - 1) // 2
    return spec.dim * b


def uci_spec(seed: int = 0, interaction: str = "dot") -> DLRMSpec:
    """UCI-health-shaped: 10 dense features, 8 tables with 2..64 rows, dim 16,
    bottom 10-32-16, top 52-32-1 (52 = 16 + C(9, 2) for the dot interaction)."""
    rng = np.random.default_rng([seed, 101])
    cards = [int(c) for c in rng.integers(2, 65, size=8)]
    s = DLRMSpec("uci", 10, [10, 32, 16], [0, 32, 1], cards, 64, 16, interaction)
    s.top[0] = top_input_width(s)
    return s


def uci_paper_spec() -> DLRMSpec:
    """The paper's UCI shape: 5 dense features and tables of [2,4,2,3,2,3,4,3] rows."""
    s = DLRMSpec("uci_paper", 5, [5, 16, 16], [0, 16, 1], [2, 4, 2, 3, 2, 3, 4, 3], 64, 16)
    s.top[0] = top_input_width(s)
    return s


def uci_silu_spec(seed: int = 0, degree: int = 7) -> DLRMSpec:
    """The UCI-shaped model with a degree-7 SiLU polynomial instead of x^2:
    three activations of depth 4 fit the 20-level chain without bootstrapping
    (ct_dense at level 18)."""
    s = uci_spec(seed)
    s.name = "uci_silu"
    s.act = silu_poly(degree)
    return s


def wide_spec(interaction: str = "dot") -> DLRMSpec:
    """A small DLRM whose packed selector is wider than 512 slots, under the
    paper's compression policy (Sec. 5.2: base 4, tables with more rows than a
    threshold compressed): tables of 700, 2000 and 3 rows with threshold 1000
    give plain one-hots of 700 and 3 slots and 6 base-4 digits (24 slots) for
    the 2000-row table, 727 slots in all; 4 dense features, bottom 4-16, top
    22-1 (22 = 16 + C(4, 2))."""
    s = DLRMSpec("wide", 4, [4, 16], [0, 1], [700, 2000, 3], 4, 16, interaction, threshold=1000)
    s.top[0] = top_input_width(s)
    return s


def wider_spec(interaction: str = "dot") -> DLRMSpec:
    """As wide_spec with a 1100-row table in place of the 700-row one: 1127
    selector slots, three ciphertexts at N = 2^10 (512 + 512 + 103 columns),
    the first two of one shape."""
    s = DLRMSpec("wider", 4, [4, 16], [0, 1], [1100, 2000, 3], 4, 16, interaction, threshold=1200)
    s.top[0] = top_input_width(s)
    return s


def criteo_cards(seed: int = 0, total: float = 33.8e6) -> list:
    """26 log-uniform cardinalities on [3, 1e7]; every k > 1e5 is multiplied by
    one common factor (clamped at 1e7), found by bisection, so the total is
    33.8M rows within 0.5%.  (The real per-feature Criteo sizes are not used.)"""
    rng = np.random.default_rng([seed, 202])
    base = np.exp(rng.uniform(np.log(3.0), np.log(1e7), size=26))
    big = base > 1e5

    def tot(f):
        k = np.where(big, np.minimum(base * f, 1e7), base)
        return np.round(k).sum()

    lo, hi = 1e-3, 1e3
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if tot(mid) < total:
            lo = mid
        else:
            hi = mid
    k = np.where(big, np.minimum(base * hi, 1e7), base)
    return [int(max(3, round(v))) for v in k]


def criteo_spec(seed: int = 0, interaction: str = "dot") -> DLRMSpec:
    """Criteo-shaped: 13 dense, 26 tables totalling ~33.8M rows, dim 16, base 64,
    bottom 13-512-256-64-16, top 367-512-256-1 (367 = 16 + C(27, 2))."""
    s = DLRMSpec("criteo", 13, [13, 512, 256, 64, 16], [0, 512, 256, 1], criteo_cards(seed), 64, 16,
                 interaction)
    s.top[0] = top_input_width(s)
    return s


def criteo_silu_boot_spec(seed: int = 0) -> DLRMSpec:
    """The Criteo-shaped model with the degree-7 SiLU fit as every activation
    (depth 4: five levels per activated layer, 34 in all), as the paper runs
    its Criteo models with polynomial activations between bootstraps (Sec.
    5.4): on the bootstrappable chain (13 compute levels) it bootstraps twice,
    before bottom layer 2 (256 slots) and on z before the interaction (512
    slots)."""
    s = criteo_spec(seed)
    s.name = "criteo_silu_boot"
    s.act = silu_poly(7)
    s.boot = ("b2", "z")
    return s


def criteo_relu_boot_spec(seed: int = 0) -> DLRMSpec:
    """The Criteo-shaped model with a degree-14 least-squares ReLU stand-in as
    every activation (relu_poly(15): powers {1, 2, 4, ..., 14}, depth 5: six
    levels per activated layer, 44 in all), as the paper runs its Criteo
    models with ReLU between bootstraps (Sec. 5.4, with composite
    polynomials and 12 bootstraps): here three bootstraps, before bottom
    layer 2 (256 slots), on z (512 slots) and before top layer 1 (512
    slots)."""
    s = criteo_spec(seed)
    s.name = "criteo_relu_boot"
    s.act = relu_poly(15)
    s.boot = ("b2", "z", "t1")
    return s


def criteo_silu_boot_fixed_spec(seed: int = 0) -> DLRMSpec:
    """criteo_silu_boot_spec with its SiLU coefficients rounded to multiples of
    2^-20 (dyadic), for the full-size parity fixture (which also fixes the
    bootstraps' cosine polynomial, spec.boot_coeffs, from its stored file)."""
    s = criteo_silu_boot_spec(seed)
    s.act = dyadic(s.act)
    return s


def uci_silu_boot_spec(seed: int = 0, boot=("b1", "z")) -> DLRMSpec:
    """A small model for the bootstrapped path: the UCI-shaped SiLU model with
    the concatenation interaction (its layout fits n = 512 slots, N = 2^10),
    bootstrapping before bottom layer 1 (32 slots) and on z (256 slots)."""
    s = uci_silu_spec(seed)
    s.name = "uci_silu_boot"
    s.interaction = "concat"
    s.top[0] = top_input_width(s)
    s.boot = tuple(boot)
    return s


def tiny_table(seed: int = 0):
    """The 1024-row x dim-16 table compressed in base 32: C_0, C_1 in U[-0.05, 0.05]^(32x16)."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(-0.05, 0.05, size=(32, 16)).astype(np.float32) for _ in range(2)]


# --------------------------------------------------------------------------
# Weights
# --------------------------------------------------------------------------
@dataclass
class DLRMWeights:
    bottom_W: list = field(default_factory=list)
    bottom_b: list = field(default_factory=list)
    top_W: list = field(default_factory=list)
    top_b: list = field(default_factory=list)
    tables: list = field(default_factory=list)      # tables[t][j]: rows x dim float32


def _calib_top_input(spec, h, embs):
    blocks = [h] + embs
    if spec.interaction == "dot":
        cols = [h]
        for a in range(len(blocks)):
            for c in range(a + 1, len(blocks)):
                cols.append(np.sum(blocks[a] * blocks[c], axis=1, keepdims=True))
        return np.concatenate(cols, axis=1)
    return np.concatenate(blocks, axis=1)


def make_weights(spec: DLRMSpec, seed: int = 0) -> DLRMWeights:
    """Weights and biases N(0, 0.1), tables U[-0.05, 0.05] (FP32), then each
    layer's (W, b) is multiplied by one scalar so its pre-activation RMS over
    256 calibration queries is 1."""
    rng = np.random.default_rng([seed, 303])
    w = DLRMWeights()
    for a, b in zip(spec.bottom[:-1], spec.bottom[1:]):
        w.bottom_W.append(rng.normal(0, 0.1, size=(b, a)))
        w.bottom_b.append(rng.normal(0, 0.1, size=b))
    for a, b in zip(spec.top[:-1], spec.top[1:]):
        w.top_W.append(rng.normal(0, 0.1, size=(b, a)))
        w.top_b.append(rng.normal(0, 0.1, size=b))
    for k in spec.cards:
        w.tables.append([rng.uniform(-0.05, 0.05, size=(r, spec.dim)).astype(np.float32)
                         for r in table_rows(k, spec.base, spec.threshold)])

    dense, idx = make_queries(spec, 256, seed=10_000 + seed)
    h = dense
    for i in range(len(w.bottom_W)):
        pre = h @ w.bottom_W[i].T + w.bottom_b[i]
        c = 1.0 / np.sqrt(np.mean(pre ** 2))
        w.bottom_W[i] *= c
        w.bottom_b[i] *= c
        h = act_apply(spec, pre * c)
    embs = []
    for t, k in enumerate(spec.cards):
        rows = table_rows(k, spec.base, spec.threshold)
        e = np.zeros((len(idx), spec.dim))
        rem = idx[:, t].astype(np.int64)
        for j, r in enumerate(rows):
            e += w.tables[t][j][rem % r].astype(np.float64)
            rem //= r
        embs.append(e)
    y = _calib_top_input(spec, h, embs)
    for i in range(len(w.top_W)):
        pre = y @ w.top_W[i].T + w.top_b[i]
        c = 1.0 / np.sqrt(np.mean(pre ** 2))
        w.top_W[i] *= c
        w.top_b[i] *= c
        y = pre * c
        if i + 1 < len(w.top_W):
            y = act_apply(spec, y)
    return w


# --------------------------------------------------------------------------
# Queries
# --------------------------------------------------------------------------
def _zipf_rank(rng, k: int, a: float = 1.1) -> int:
    while True:
        r = int(rng.zipf(a))
        if r <= k:
            return r


def make_queries(spec: DLRMSpec, count: int, seed: int = 0):
    """(dense [count, n_dense] float64, indices [count, T] uint64).

    UCI-shaped dense features are N(0,1) with uniform indices; Criteo-shaped
    dense features are log(1 + x), x ~ LogNormal(0,1) (heavy-tailed counts
    through the logarithm DLRM pipelines apply to Criteo's count features),
    with Zipf(1.1) ranks mapped to rows by a seeded affine bijection
    r -> (a r + c) mod k, gcd(a, k) = 1."""
    rng = np.random.default_rng([seed, 404])
    T = len(spec.cards)
    if spec.name.startswith("criteo"):
        dense = np.log1p(rng.lognormal(0.0, 1.0, size=(count, spec.n_dense)))
        prm = np.random.default_rng([seed, 405])
        idx = np.zeros((count, T), dtype=np.uint64)
        for t, k in enumerate(spec.cards):
            a = int(prm.integers(1, max(k, 2)))
            while np.gcd(a, k) != 1:
                a += 1
            c = int(prm.integers(0, k))
            for q in range(count):
                r = _zipf_rank(rng, k) - 1
                idx[q, t] = (a * r + c) % k
    else:
        dense = rng.normal(0.0, 1.0, size=(count, spec.n_dense))
        idx = np.stack([rng.integers(0, k, size=count) for k in spec.cards], axis=1).astype(np.uint64)
    return dense, idx


# --------------------------------------------------------------------------
# Serving traces
# --------------------------------------------------------------------------
def serving_trace(rate: float, count: int, n_uci_clients: int, n_criteo_clients: int, frac_uci: float = 0.8,
                  seed: int = 0):
    """Poisson arrivals at `rate` requests/s: (arrival_s [count] sorted,
    client [count]).  A request is UCI-shaped with probability frac_uci (its
    client uniform among clients 0..n_uci_clients-1), else Criteo-shaped
    (client uniform among the next n_criteo_clients)."""
    rng = np.random.default_rng([seed, 505])
    arrival = np.cumsum(rng.exponential(1.0 / rate, size=count))
    arrival -= arrival[0]
    uci = rng.random(count) < frac_uci
    client = np.where(uci, rng.integers(0, n_uci_clients, count),
                      n_uci_clients + rng.integers(0, n_criteo_clients, count))
    return arrival, client.astype(np.uint32)


# --------------------------------------------------------------------------
# Platform-independent integer inputs (full-size parity fixtures)
# --------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (Steele, Lea, Flood 2014) on uint64
    arrays, wrapping arithmetic."""
    with np.errstate(over="ignore"):
        z = x.copy()
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def int_poly(seed: int, index: int, n: int, bound: int = 1 << 20) -> np.ndarray:
    """n signed integers in [-bound, bound], a pure function of (seed, index):
    SplitMix64 of the counters (seed, index, j), reduced mod 2 bound + 1.
    Integer-only, so it gives the same values on every machine and numpy
    version (the FP64 encoder does not: its last-bit rounding can differ)."""
    with np.errstate(over="ignore"):
        base = _splitmix64(np.array([(seed & (2**64 - 1)) ^ 0x5DEECE66D], dtype=np.uint64))[0]
        base = _splitmix64(np.array([base ^ np.uint64(index & (2**64 - 1))], dtype=np.uint64))[0]
        ctr = base + (np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN)
    z = _splitmix64(ctr)
    m = np.uint64(2 * bound + 1)
    return (z % m).astype(np.int64) - bound


def dyadic(coeffs, bits: int = 20) -> tuple:
    """Coefficients rounded to multiples of 2^-bits: exact binary fractions,
    so a model built from them is the same on every machine (a least-squares
    fit's last bits depend on the linear-algebra library)."""
    return tuple(float(np.round(float(a) * 2.0**bits)) / 2.0**bits for a in coeffs)


def uci_silu_fixed_spec(seed: int = 0) -> DLRMSpec:
    """uci_silu_spec with its SiLU coefficients rounded to multiples of 2^-20
    (dyadic), for the full-size parity fixtures."""
    s = uci_silu_spec(seed)
    s.act = dyadic(s.act)
    return s
