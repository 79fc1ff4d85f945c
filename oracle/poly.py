"""Homomorphic evaluation of a real polynomial on a CKKS ciphertext (test
infrastructure only: tests, smoke() and bench's CPU leg use it).

The paper's Criteo models use polynomial approximations of ReLU and SiLU as
activations (Sec. 2.1.4 and Sec. 5.4: composite ReLU polynomials and a
lower-degree SiLU), evaluated homomorphically with ct x ct products and
constant multiplications.  The paper prints neither the coefficients nor the
evaluation schedule, so the schedule below is a reading, fixed for both sides:

  - powers: x^1 = x; x^k = x^a * x^(k-a) with a the largest power of two
    below k (a ct x ct product: tensor, relinearise, rescale; operands taken
    to the lower of their two levels first), so x^k sits ceil(log2 k) levels
    below x.  Only the powers a non-zero a_k needs are formed: the k >= 1
    with a_k != 0 and, recursively, the operands of their products, in
    increasing k;
  - terms: every x^k with a_k != 0 is taken to the level L_c of the deepest
    power and multiplied by the integer c_k = round_half_away(a_k * s_k),
    s_k = (target_scale * q_{L_c}) / scale(x^k), so all terms carry the scale
    target_scale * q_{L_c} (up to FP64 rounding of s_k) and add exactly;
  - the sum is rescaled once (scale ~ target_scale, level L_c - 1) and a_0
    is added as the integer round_half_away(a_0 * scale) in coefficient 0.

The evaluation therefore consumes ceil(log2 d) + 1 levels for d >= 2 (one
level for d = 1).  Every step is an exact integer operation except the FP64
products that fix the constants, which both implementations form in the
same order.
"""
from __future__ import annotations

import math

import numpy as np

from . import ckks, ring


def operands(k: int):
    """x^k = x^a * x^b: a the largest power of two below k, b = k - a."""
    a = 1 << ((k - 1).bit_length() - 1)
    return a, k - a


def product_tree(coeffs):
    """[(k, a, b)] in increasing k: the products that form every power a
    non-zero coefficient of degree >= 2 needs."""
    need = set()

    def want(k):
        if k >= 2 and k not in need:
            need.add(k)
            for j in operands(k):
                want(j)

    for k in range(2, len(coeffs)):
        if coeffs[k] != 0:
            want(k)
    return [(k, *operands(k)) for k in sorted(need)]


def power_depth(k: int) -> int:
    """Levels x^k sits below x: ceil(log2 k)."""
    return (k - 1).bit_length()


def depth(d: int) -> int:
    """Levels the whole evaluation consumes (powers, then one for the constants)."""
    return 0 if d == 0 else power_depth(d) + 1


def round_half_away(v: float) -> int:
    return int(math.copysign(math.floor(abs(v) + 0.5), v))


def mul_int(p: ckks.Params, a: ckks.Ct, c: int, factor: float) -> ckks.Ct:
    """a * c for an integer c (mod every q of the level); the declared scale
    becomes a.scale * factor."""
    mods = p.q_mods(a.level)
    cs = [c % q for q in mods]
    return ckks.Ct(ring.mul_scalar(a.c0, cs, mods), ring.mul_scalar(a.c1, cs, mods), a.level, a.scale * factor)


def add_int(p: ckks.Params, a: ckks.Ct, c: int) -> ckks.Ct:
    """a + c, the integer c in coefficient 0 of the plaintext (a constant in every slot)."""
    mods = p.q_mods(a.level)
    if abs(c) >= 2**63:
        raise ValueError("constant too large")
    m = np.zeros(p.N, dtype=np.int64)
    m[0] = c
    return ckks.Ct(ring.add(a.c0, ring.from_signed(m, mods), mods), a.c1.copy(), a.level, a.scale)


def simulate(q, level: int, scale: float, coeffs, target_scale: float):
    """(output level, output scale) of poly_eval on a ciphertext at (level,
    scale), from the same FP64 steps; q: the chain's primes."""
    lv, sc = {1: level}, {1: scale}
    for k, a, b in product_tree(coeffs):
        lv[k] = min(lv[a], lv[b])
        sc[k] = (sc[a] * sc[b]) / float(q[lv[k]])
        lv[k] -= 1
    d = len(coeffs) - 1
    level_c = level - power_depth(d)
    first = next(k for k in range(1, d + 1) if coeffs[k] != 0)
    s = (target_scale * float(q[level_c])) / sc[first]
    return level_c - 1, (sc[first] * s) / float(q[level_c])


def term_constants(x_scale_by_power: dict, level_c: int, p: ckks.Params, coeffs, target_scale: float):
    """[(k, c_k, s_k)] for the non-zero a_k, k >= 1 (the FP64 steps of the reading)."""
    out = []
    for k in range(1, len(coeffs)):
        if coeffs[k] == 0:
            continue
        s = (target_scale * float(p.q[level_c])) / x_scale_by_power[k]
        out.append((k, round_half_away(float(coeffs[k]) * s), s))
    return out


def poly_eval(p: ckks.Params, keys: ckks.Keys, x: ckks.Ct, coeffs, target_scale: float) -> ckks.Ct:
    """sum_k coeffs[k] x^k on the slots of x (degree d = len(coeffs) - 1 >= 1,
    at least one non-zero coefficient of degree >= 1)."""
    d = len(coeffs) - 1
    if d < 1 or coeffs[d] == 0 or not any(coeffs[1:]):
        raise ValueError("need a non-constant polynomial with a non-zero leading coefficient")
    if x.level < depth(d):
        raise ValueError("not enough levels for this degree")
    pw = {1: x}
    for k, a, b in product_tree(coeffs):
        lvl = min(pw[a].level, pw[b].level)
        pw[k] = ckks.mul(p, keys, ckks.drop_level(p, pw[a], lvl), ckks.drop_level(p, pw[b], lvl))
    level_c = x.level - power_depth(d)
    acc = None
    for k, c, s in term_constants({k: pw[k].scale for k in pw}, level_c, p, coeffs, target_scale):
        t = mul_int(p, ckks.drop_level(p, pw[k], level_c), c, s)
        acc = t if acc is None else ckks.add(p, acc, t)
    y = ckks.rescale(p, acc)
    if coeffs[0] != 0:
        y = add_int(p, y, round_half_away(float(coeffs[0]) * y.scale))
    return y
