"""CKKS bootstrapping of sparsely packed real slots (test infrastructure only:
tests, smoke() and bench's CPU leg use it).

The paper refreshes the level of a ciphertext by bootstrapping (Sec. 2.1.4;
its Criteo models with ReLU or SiLU activations need 12 or 5 of them,
Sec. 5.4) and names its parts (ModRaise, CoeffToSlot, EvalMod, SlotToCoeff)
without giving their steps.  The reading here (fixed for both sides) is the
standard pipeline for a ciphertext whose real slot vector is periodic with
period n_s (2 n_s <= n = N/2), under a secret with h non-zero coefficients:

  1. boost: at level 0 the ciphertext is multiplied by the integer 2^b, so
     the message m = 2^b * scale * z stays a small fraction of q_0;
  2. ModRaise: c0 and c1 (mod q_0, centred) are read as integers modulo
     every prime of the top level L; the ciphertext now decrypts to
     m + q_0 I over Q_L, I an integer polynomial, |I_k| <= (h + 1) / 2;
  3. SubSum: ct += rot(ct, n_s 2^i) for i < log2(n / n_s).  This is the
     trace onto Z[Y], Y = X^g, g = N / (2 n_s): it keeps g times the
     coefficients at multiples of g and cancels the others;
  4. CoeffToSlot: the 2 n_s coefficients t_k of the polynomial in Y and its
     n_s slot values w_i are tied by w = U t, U[i, k] = xi^(k 5^i),
     xi = exp(i pi / (2 n_s)), so t = (U^H w + U^T conj(w)) / (2 n_s).  The
     second term is the conjugate of the first (U^T conj(w) = conj(U^H w)),
     so one BSGS matvec C = U^H w / (2 n_s) and the conjugate of its output
     give t = C + conj(C); the slots (period 2 n_s) then hold u_k / 2^r,
     u_k = m_k / q_0 + I_k, at about eval_scale.  The diagonals are encoded at eval_scale times the
     primes the product is rescaled by, over q_0: one rescale when the top
     primes are 60-bit (the bootstrappable chain), two on an all-40-bit
     chain, so that their rounding stays below the noise;
  5. EvalMod: y = u / 2^r - 1 / (4 2^r) (a constant), c = p(y), p a
     polynomial fit of cos(2 pi y) on |y| <= (K + 1/2) / 2^r (even degree),
     then r double angles c <- 2 c^2 - 1, so c = cos(2 pi (u - 1/4)) =
     sin(2 pi u) = sin(2 pi m_k / q_0), about 2 pi m_k / q_0;
  6. SlotToCoeff: z = U (q_0 / (2 pi 2^b s_ref)) c, a BSGS matvec from
     period 2 n_s to period n_s (one fold): the slots hold the message again.

EvalMod runs at eval_scale (about its primes: 2^60 on the bootstrappable
chain, whose top 13 primes are 60-bit, so its noise stays far below the
message after the r double angles multiply it).  The output sits
cts_levels + depth(p) + r + 1 levels below L (poly.depth), at a scale about
Delta.  Every step is an exact integer operation of ckks / linear /
poly; only the constants (diagonals, polynomial, the scales) come from FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import ckks, linear, poly, ring


@dataclass
class BootParams:
    n_s: int                     # slot period of the input and output (power of two, 2 n_s <= n)
    K: int = 24                  # |I_k| the sine must cover (about 6 sigma for h = 192)
    r: int = 6                   # double angles
    degree: int = 16             # even degree of the cosine fit
    log2_boost: int = 10         # the message is multiplied by 2^b at level 0
    s_ref: float = 2.0**40       # the input scale the SlotToCoeff constants assume
    cts_levels: int = 1          # rescales after CoeffToSlot (2 when the top primes are small)
    eval_scale: float = 2.0**60  # the scale EvalMod runs at (about its primes)
    coeffs: list | None = None   # the cosine polynomial (power basis in y); None: cos_fit


def slot_matrix(n_s: int) -> np.ndarray:
    """U[i, k] = xi^(k 5^i mod 4 n_s), xi = exp(i pi / (2 n_s)): n_s x 2 n_s.
    The slots of a polynomial sum_k t_k Y^k (Y = X^(N/(2 n_s))) are U t."""
    e = np.array([pow(5, i, 4 * n_s) for i in range(n_s)], dtype=np.int64)
    k = np.arange(2 * n_s, dtype=np.int64)
    return np.exp(1j * np.pi * ((np.outer(e, k)) % (4 * n_s)) / (2 * n_s))


def cos_fit(K: int, r: int, degree: int) -> list:
    """Power-basis coefficients (in y) of the interpolant of cos(2 pi y) at
    the degree + 1 Chebyshev nodes of [-Y, Y], Y = (K + 1/2) / 2^r; the odd
    coefficients (zero for an even function) are set to exact zeros."""
    if degree < 2 or degree % 2:
        raise ValueError("the cosine fit needs an even degree >= 2")
    Y = (K + 0.5) / 2.0**r
    ch = np.polynomial.Chebyshev.interpolate(lambda y: np.cos(2 * np.pi * y), degree, domain=[-Y, Y])
    c = ch.convert(kind=np.polynomial.Polynomial, domain=[-1.0, 1.0], window=[-1.0, 1.0]).coef
    c = [float(v) for v in c] + [0.0] * (degree + 1 - len(c))
    for k in range(1, degree + 1, 2):
        c[k] = 0.0
    return c


def levels_used(bp: BootParams) -> int:
    """Levels between the top of the chain and the output."""
    return bp.cts_levels + poly.depth(bp.degree) + bp.r + 1


@dataclass
class Boot:
    bp: BootParams
    g: int                       # N / (2 n_s)
    level_top: int
    cts: list                    # [A]: the CoeffToSlot PtMatrix, at level L
    stc: linear.PtMatrix
    coeffs: list
    subsum_steps: list = field(default_factory=list)

    def rotation_steps(self) -> list:
        st = set(self.subsum_steps)
        for pm in self.cts + [self.stc]:
            st |= set(linear.rotation_steps(pm))
        return sorted(st)


def prepare(p: ckks.Params, bp: BootParams) -> Boot:
    n_s = bp.n_s
    if n_s < 1 or n_s & (n_s - 1) or 2 * n_s > p.n:
        raise ValueError("n_s must be a power of two with 2 n_s <= n")
    L = p.L
    if levels_used(bp) > L:
        raise ValueError("the chain is too short for this bootstrapping")
    g = p.N // (2 * n_s)
    U = slot_matrix(n_s)
    # CoeffToSlot at level L: inputs read at scale q_0 (values g U u), outputs
    # u / 2^r at about eval_scale after cts_levels rescales
    f = 1.0 / (2 * n_s * g * 2.0**bp.r)
    pt_cts = bp.eval_scale
    for i in range(bp.cts_levels):
        pt_cts *= float(p.q[L - i])
    pt_cts /= float(p.q[0])
    out_cts = float(p.q[0]) * pt_cts / float(p.q[L])
    A = linear.prepare_scaled(p, f * U.conj().T, n_s, 2 * n_s, L, pt_cts, out_cts)
    # SlotToCoeff at the level EvalMod ends on: from about eval_scale to Delta
    ls = L - levels_used(bp) + 1
    S = (float(p.q[0]) / (2 * math.pi * 2.0**bp.log2_boost * bp.s_ref)) * U
    stc = linear.prepare_scaled(p, S, 2 * n_s, n_s, ls, float(p.q[ls]) * p.delta / bp.eval_scale, p.delta)
    coeffs = list(bp.coeffs) if bp.coeffs is not None else cos_fit(bp.K, bp.r, bp.degree)
    steps = [n_s << i for i in range((p.n // n_s).bit_length() - 1)]
    return Boot(bp, g, L, [A], stc, coeffs, steps)


def scales(p: ckks.Params, boot: Boot):
    """(CoeffToSlot output scale, EvalMod output scale): the scales the run
    declares, from the same FP64 steps (they do not depend on the input)."""
    s, lv = boot.cts[0].out_scale, boot.level_top - 1
    for _ in range(boot.bp.cts_levels - 1):
        s = s / float(p.q[lv])
        lv -= 1
    lv2, s2 = poly.simulate(p.q, lv, s, boot.coeffs, boot.bp.eval_scale)
    for _ in range(boot.bp.r):
        s2 = (s2 * s2) / float(p.q[lv2])
        lv2 -= 1
    return s, s2


def out_scale(p: ckks.Params, boot: Boot, in_scale: float) -> float:
    """The declared scale of the output for an input of scale in_scale."""
    s2 = scales(p, boot)[1]
    return (s2 * boot.stc.pt_scale) / float(p.q[boot.stc.level]) * (in_scale / boot.bp.s_ref)


def mod_raise(p: ckks.Params, ct: ckks.Ct) -> ckks.Ct:
    """A level-0 ciphertext read as centred integers modulo every prime of
    the top level (declared scale q_0: the values are then (m + q_0 I) / q_0)."""
    if ct.level != 0:
        raise ValueError("ModRaise takes a level-0 ciphertext")
    q0 = int(p.q[0])
    mods = p.q_mods(p.L)

    def lift(a):
        v = a[0].astype(np.int64)
        v = np.where(a[0] > np.uint64((q0 - 1) // 2), v - np.int64(q0), v)   # centred in (-q0/2, q0/2]
        return ring.from_signed(v, mods)

    return ckks.Ct(lift(ct.c0), lift(ct.c1), p.L, float(p.q[0]))


def subsum(p: ckks.Params, keys: ckks.Keys, ct: ckks.Ct, steps) -> ckks.Ct:
    for st in steps:
        ct = ckks.add(p, ct, ckks.rotate(p, keys, ct, st))
    return ct


def coeff_to_slot(p: ckks.Params, keys: ckks.Keys, boot: Boot, ct: ckks.Ct) -> ckks.Ct:
    y = linear.matvec(p, keys, boot.cts[0], ct)
    y = ckks.add(p, y, ckks.conjugate(p, keys, y))
    for _ in range(boot.bp.cts_levels - 1):
        y = ckks.rescale(p, y)
    return y


def eval_mod(p: ckks.Params, keys: ckks.Keys, boot: Boot, y: ckks.Ct) -> ckks.Ct:
    r = boot.bp.r
    y = poly.add_int(p, y, poly.round_half_away(-y.scale / (4.0 * 2.0**r)))
    c = poly.poly_eval(p, keys, y, boot.coeffs, boot.bp.eval_scale)
    for _ in range(r):
        c = ckks.mul(p, keys, c, c)
        c = ckks.add(p, c, c)
        c = poly.add_int(p, c, poly.round_half_away(-c.scale))
    return c


def slot_to_coeff(p: ckks.Params, keys: ckks.Keys, boot: Boot, c: ckks.Ct, in_scale: float) -> ckks.Ct:
    """The StC product; its declared scale is the product's (c.scale times
    the diagonals' scale, over q_l) times in_scale / s_ref, so the slots
    decode to the input's values."""
    z = linear.matvec(p, keys, boot.stc, c)
    z.scale = (c.scale * boot.stc.pt_scale) / float(p.q[boot.stc.level]) * (in_scale / boot.bp.s_ref)
    return z


def boost(p: ckks.Params, ct: ckks.Ct, log2_boost: int) -> ckks.Ct:
    """Drop to level 0 and multiply by the integer 2^b (scale times 2^b)."""
    ct = ckks.drop_level(p, ct, 0)
    return poly.mul_int(p, ct, 1 << log2_boost, 2.0**log2_boost)


def bootstrap(p: ckks.Params, keys: ckks.Keys, boot: Boot, ct: ckks.Ct, stages: dict | None = None) -> ckks.Ct:
    """The whole pipeline; `stages`, if given, receives every intermediate ciphertext."""
    in_scale = ct.scale
    x = boost(p, ct, boot.bp.log2_boost)
    x = mod_raise(p, x)
    if stages is not None:
        stages["raised"] = x
    x = subsum(p, keys, x, boot.subsum_steps)
    if stages is not None:
        stages["subsum"] = x
    y = coeff_to_slot(p, keys, boot, x)
    if stages is not None:
        stages["cts"] = y
    c = eval_mod(p, keys, boot, y)
    if stages is not None:
        stages["evalmod"] = c
    z = slot_to_coeff(p, keys, boot, c, in_scale)
    if stages is not None:
        stages["out"] = z
    return z
