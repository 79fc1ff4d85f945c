"""Prime chain and roots of unity for RNS-CKKS (test infrastructure only).

The paper fixes Q = prod q_i with word-sized primes (appendix "CKKS
operations") but not how they are chosen.  The reading used on both sides:
every prime is NTT-friendly (q = 1 mod 2N); for each requested bit size the
primes are the largest such ones below 2^bits, in decreasing order, never
reusing a prime already taken.  The ciphertext primes q_0..q_L are chosen
first, in their listed order, then the K special primes (all of
``p_bits``).  Primality is deterministic Miller-Rabin with the twelve prime
bases 2..37, which is exact below 3.3e24 > 2^64.
"""
from __future__ import annotations

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(bits: int, count: int, two_n: int, exclude=()) -> list[int]:
    """The `count` largest primes q < 2^bits with q = 1 mod two_n, not in exclude."""
    out = []
    c = ((2**bits - 1) // two_n) * two_n + 1
    if c >= 2**bits:
        c -= two_n
    while len(out) < count:
        if c < 2 ** (bits - 1):
            raise ValueError(f"not enough {bits}-bit primes = 1 mod {two_n}")
        if c not in exclude and is_prime(c):
            out.append(c)
        c -= two_n
    return out


def prime_chain(log_n: int, q_bits, n_p: int, p_bits: int):
    """(q list, p list) for ring degree 2^log_n."""
    two_n = 2 << log_n
    qs: list[int] = []
    for b in q_bits:
        qs += ntt_primes(b, 1, two_n, exclude=set(qs))
    ps = ntt_primes(p_bits, n_p, two_n, exclude=set(qs))
    return qs, ps


def smallest_non_residue(q: int) -> int:
    """Smallest g > 1 with g^((q-1)/2) = -1 mod q (Euler's criterion)."""
    g = 2
    while pow(g, (q - 1) // 2, q) != q - 1:
        g += 1
    return g


def primitive_2n_root(q: int, two_n: int) -> int:
    """psi = g^((q-1)/2N) for the smallest quadratic non-residue g.

    A non-residue generates the full 2-power part of Z_q^*, so psi has order
    exactly 2N: psi^N = -1.
    """
    g = smallest_non_residue(q)
    psi = pow(g, (q - 1) // two_n, q)
    assert pow(psi, two_n // 2, q) == q - 1
    return psi
