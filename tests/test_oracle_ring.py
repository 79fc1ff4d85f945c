"""Pins for the oracle's ring arithmetic: 128-bit modmul, primes and roots,
schoolbook and NTT negacyclic products (all checked against definitions that
do not share code with the oracle: Python big integers, sympy, brute force)."""
import random

import numpy as np
import pytest

from oracle import primes, ring


def py_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


def test_mul_mod_matches_big_integers():
    rnd = random.Random(1)
    for q in [2**61 - 1, (1 << 40) - 87, 1152921504606830593, 3]:
        cases = [(0, 0), (q - 1, q - 1), (q - 1, 1), (2**64 - 1, 2**64 - 1), (2**64 - 1, q - 1)]
        cases += [(rnd.randrange(2**64), rnd.randrange(2**64)) for _ in range(200)]
        for a, b in cases:
            assert ring.lib().orc_mul_mod(a, b, q) == (a * b) % q


def test_miller_rabin_agrees_with_sympy():
    sympy = pytest.importorskip("sympy")
    rnd = random.Random(2)
    nums = [rnd.randrange(2**64) | 1 for _ in range(3000)] + [2, 3, 4, 561, 1105, 2**61 - 1]
    # strong pseudoprimes to several small bases
    nums += [3215031751, 2152302898747, 3474749660383, 341550071728321, 3825123056546413051]
    for x in nums:
        assert primes.is_prime(x) == bool(sympy.isprime(x)), x


@pytest.mark.parametrize("log_n,q_bits,n_p,p_bits", [
    (16, [60] + [40] * 20, 3, 60),
    (13, [50, 50, 50], 1, 50),
])
def test_prime_chain_is_the_largest_ntt_primes(log_n, q_bits, n_p, p_bits):
    sympy = pytest.importorskip("sympy")
    qs, ps = primes.prime_chain(log_n, q_bits, n_p, p_bits)
    two_n = 2 << log_n
    allp = qs + ps
    assert len(set(allp)) == len(allp)
    for x, b in zip(allp, q_bits + [p_bits] * n_p):
        assert sympy.isprime(x) and x % two_n == 1 and x < 2**b and x > 2 ** (b - 1)
    # For each bit size, the chosen primes are exactly the largest ones.
    for b in set(q_bits + [p_bits]):
        chosen = sorted([x for x in allp if x.bit_length() == b], reverse=True)
        c = ((2**b - 1) // two_n) * two_n + 1
        found = []
        while len(found) < len(chosen):
            if sympy.isprime(c):
                found.append(c)
            c -= two_n
        assert found == chosen
    # order: q_0 is the largest of its size, then q_1 > q_2 > ... within a size
    assert qs[0] == max(x for x in allp if x.bit_length() == q_bits[0])


def test_primitive_root_has_order_2n():
    for q in primes.ntt_primes(40, 3, 2**17) + primes.ntt_primes(60, 2, 2**14):
        two_n = 2**17 if q.bit_length() == 40 else 2**14
        psi = primes.primitive_2n_root(q, two_n)
        assert pow(psi, two_n, q) == 1 and pow(psi, two_n // 2, q) == q - 1
        g = primes.smallest_non_residue(q)
        assert all(pow(h, (q - 1) // 2, q) == 1 for h in range(2, g))


@pytest.fixture(scope="module")
def pq():
    out = []
    for bits, n in [(40, 1024), (60, 1024), (50, 8192)]:
        q = primes.ntt_primes(bits, 1, 2 * n)[0]
        out.append((q, n, primes.primitive_2n_root(q, 2 * n)))
    return out


def test_schoolbook_matches_python_brute_force():
    q = primes.ntt_primes(60, 1, 32)[0]
    rng = np.random.default_rng(3)
    for n in [1, 2, 4, 16]:
        a = rng.integers(0, q, n, dtype=np.uint64)
        b = rng.integers(0, q, n, dtype=np.uint64)
        assert [int(x) for x in ring.schoolbook(a, b, q)] == py_negacyclic(a, b, q)


def test_x_pow_n_is_minus_one():
    q = primes.ntt_primes(50, 1, 64)[0]
    n = 32
    a = np.zeros(n, dtype=np.uint64)
    b = np.zeros(n, dtype=np.uint64)
    a[n - 1] = 1
    b[1] = 1                                     # X^(N-1) * X = X^N = -1
    out = ring.schoolbook(a, b, q)
    assert int(out[0]) == q - 1 and not np.any(out[1:])


def test_ntt_forward_is_evaluation_at_odd_powers(pq):
    q, _, _ = pq[0]
    n = 64
    psi = primes.primitive_2n_root(q, 2 * n)
    rng = np.random.default_rng(4)
    a = rng.integers(0, q, n, dtype=np.uint64)
    ah = ring.ntt(a, [q], [psi])[0]
    for k in range(n):
        x = pow(psi, 2 * k + 1, q)
        val = 0
        for c in reversed([int(v) for v in a]):       # Horner
            val = (val * x + c) % q
        assert int(ah[k]) == val


def test_ntt_round_trip_and_product_equals_schoolbook(pq):
    rng = np.random.default_rng(5)
    for q, n, psi in pq:
        a = rng.integers(0, q, (2, n), dtype=np.uint64)
        b = rng.integers(0, q, (2, n), dtype=np.uint64)
        back = ring.ntt(ring.ntt(a, [q, q], [psi, psi]), [q, q], [psi, psi], inverse=True)
        assert np.array_equal(back, a)
        if n <= 1024:
            prod = ring.polymul(a, b, [q, q], [psi, psi])
            for l in range(2):
                assert np.array_equal(prod[l], ring.schoolbook(a[l], b[l], q))


def test_ntt_product_equals_schoolbook_at_8192(pq):
    q, n, psi = pq[2]
    rng = np.random.default_rng(6)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = np.zeros(n, dtype=np.uint64)
    b[rng.integers(0, n, 6)] = rng.integers(0, q, 6, dtype=np.uint64)   # sparse: fast brute force
    want = np.zeros(n, dtype=object)
    for j in np.nonzero(b)[0]:
        for i in range(n):
            k = i + j
            v = int(a[i]) * int(b[j])
            if k < n:
                want[k] += v
            else:
                want[k - n] -= v
    want = [int(x) % q for x in want]
    got = ring.polymul(a, b, [q], [psi])[0]
    assert [int(x) for x in got] == want


def test_reduce128_and_scalar_ops():
    q = primes.ntt_primes(40, 1, 2048)[0]
    rng = np.random.default_rng(7)
    hi = rng.integers(0, 2**63, 100, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    lo = rng.integers(0, 2**63, 100, dtype=np.uint64)
    got = ring.reduce128(hi, lo, [q])[0]
    assert [int(x) for x in got] == [((int(h) << 64) | int(l)) % q for h, l in zip(hi, lo)]
    c = 123456789123456789
    got = ring.mul_scalar(hi, [c], [q])[0]
    assert [int(x) for x in got] == [int(h) * (c % q) % q for h in hi]


def test_exact_mode_gives_the_same_products_and_matvec():
    """ckks.EXACT (every ring product by the O(N^2) schoolbook convolution)
    changes no result: a product and a whole BSGS matvec with folds agree
    word for word with the NTT path."""
    from oracle import ckks, linear
    p = ckks.Params(8, [60, 40, 40], 3, 60, 3, 40.0)
    rng = np.random.default_rng(5)
    a = np.stack([rng.integers(0, q, p.N, dtype=np.uint64) for q in p.q])
    b = np.stack([rng.integers(0, q, p.N, dtype=np.uint64) for q in p.q])
    W = rng.normal(0, 0.3, (4, 16))
    pm = linear.prepare(p, W, 16, 4, 2, p.delta, p.delta)
    sk, keys = ckks.keygen(p, 3, rot_steps=linear.rotation_steps(pm))
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, rng.uniform(-1, 1, p.n), p.delta), 2, p.delta, 9)
    fast_prod, fast_mv = ckks.polymul(p, a, b, p.q), linear.matvec(p, keys, pm, ct)
    try:
        ckks.EXACT = True
        exact_prod, exact_mv = ckks.polymul(p, a, b, p.q), linear.matvec(p, keys, pm, ct)
    finally:
        ckks.EXACT = False
    assert np.array_equal(fast_prod, exact_prod)
    assert np.array_equal(fast_mv.c0, exact_mv.c0) and np.array_equal(fast_mv.c1, exact_mv.c1)
