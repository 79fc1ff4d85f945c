"""Plaintext-matrix x ciphertext-vector products (test infrastructure only).

Halevi-Shoup diagonal method and its baby-step giant-step (BSGS) form
(HE-LRM Sec. 2.1.4 "Neural Network Layers in FHE": the diagonals of the weight
matrix multiply rotations of the input; BSGS pre-rotates the diagonals so only
O(sqrt n) rotations remain), evaluated with double hoisting (Sec. 3.2.1 cites
the double-hoisted BSGS of Bossuat et al.: one ModUp shared by the baby steps,
products accumulated over QP, the giant-step rotations applied to QP
ciphertexts, one final ModDown).

Layout (a reading: the paper shows it only in a figure).  A vector of padded
length v = 2^k is replicated with period v over all n slots.  For a matrix
n_out x n_in padded to out_pad x in_pad (powers of two) there are
D = min(in_pad, out_pad) extended diagonals

    diag_i[j] = W[j mod out_pad, (j + i) mod in_pad],   j < n,  i < D,

and, when in_pad > out_pad, the folds: sum_j rot(y, j out_pad) over j <
in_pad / out_pad, in levels of up to 3 hoisted rotations (fold_plan).
The result is W x replicated with period out_pad.  BSGS split: n1 =
min(D, max(16, D / 8)), n2 = D / n1 (see bsgs_split); i = g*n1 + b and
diag'_{g,b} = rot(diag_{g n1 + b}, -g n1).  All-zero diagonals are skipped,
which changes no result (their products are exactly zero).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ckks, ring


def pow2ceil(x: int) -> int:
    x = max(int(x), 1)
    return 1 << (x - 1).bit_length()


BABY_MIN, GIANT_MAX = 16, 8


def bsgs_split(D: int):
    """n1 = min(D, max(16, D / 8)) baby steps, n2 = D / n1 giant steps.

    The paper fixes only that BSGS needs O(sqrt n) rotations, not the split.
    A hoisted baby step costs one key inner product (a key read), a giant
    step a ModDown and a ModUp as well; this split keeps at most 8 giant
    steps and otherwise trades baby-step keys for giant steps."""
    n1 = min(D, max(BABY_MIN, D // GIANT_MAX))
    return n1, D // n1


def extended_diagonals(W: np.ndarray, in_pad: int, out_pad: int, n: int) -> np.ndarray:
    """[D, n] array of diag_i[j] = Wpad[j mod out_pad, (j+i) mod in_pad] (float64, or complex128 for a complex W)."""
    Wp = np.zeros((out_pad, in_pad), dtype=np.result_type(W.dtype, np.float64))
    Wp[: W.shape[0], : W.shape[1]] = W
    D = min(in_pad, out_pad)
    j = np.arange(n)
    return np.stack([Wp[j % out_pad, (j + i) % in_pad] for i in range(D)])


FOLD_RADIX_BITS = 2


def fold_plan(in_pad: int, out_pad: int):
    """The folds of a wide matrix as levels [(stride, radix)], from the
    smallest stride: level t adds rot(y, d * stride_t) for d = 1..radix_t - 1
    (hoisted rotations of the same ciphertext), radix 4 except the last, so
    that together they sum rot(y, j * out_pad) over j < in_pad / out_pad."""
    bits = (in_pad // out_pad).bit_length() - 1
    out, stride = [], out_pad
    while bits > 0:
        r = min(FOLD_RADIX_BITS, bits)
        out.append((stride, 1 << r))
        stride <<= r
        bits -= r
    return out


def fold_steps(folds):
    return [d * s for s, r in folds for d in range(1, r)]


@dataclass
class Layout:
    in_pad: int
    out_pad: int
    D: int
    n1: int
    n2: int
    folds: list

    @staticmethod
    def make(in_pad: int, out_pad: int) -> "Layout":
        D = min(in_pad, out_pad)
        n1, n2 = bsgs_split(D)
        return Layout(in_pad, out_pad, D, n1, n2, fold_plan(in_pad, out_pad))


@dataclass
class PtMatrix:
    """Encoded pre-rotated diagonals of one layer at input level `level`.

    `pts` maps (g, b) -> signed integer coefficients (length N) for the
    non-zero diagonals, listed in (g, b) order; `pt_scale` is their scale.
    """
    layout: Layout
    level: int
    pt_scale: float
    out_scale: float
    pts: dict = field(default_factory=dict)

    def ordered_keys(self):
        return sorted(self.pts)


def prepare(p: ckks.Params, W: np.ndarray, in_pad: int, out_pad: int, level: int,
            ct_scale: float, target_scale: float) -> PtMatrix:
    """Encode the diagonals so the rescaled output has scale exactly target_scale:
    pt_scale = q_l * target / ct_scale."""
    pt_scale = float(p.q[level]) * target_scale / ct_scale
    return prepare_scaled(p, np.asarray(W, dtype=np.float64), in_pad, out_pad, level, pt_scale, target_scale)


def prepare_scaled(p: ckks.Params, W: np.ndarray, in_pad: int, out_pad: int, level: int,
                   pt_scale: float, out_scale: float) -> PtMatrix:
    """The diagonals of a real or complex W encoded at pt_scale; out_scale is
    the scale the product declares after its rescale."""
    lay = Layout.make(in_pad, out_pad)
    W = np.asarray(W)
    diags = extended_diagonals(W, in_pad, out_pad, p.n)
    enc = ckks.encode_complex if np.iscomplexobj(W) else ckks.encode_real
    pm = PtMatrix(lay, level, pt_scale, out_scale)
    for g in range(lay.n2):
        for b in range(lay.n1):
            dg = diags[g * lay.n1 + b]
            if not np.any(dg):
                continue
            rot = np.roll(dg, g * lay.n1)            # rot(x, -s)[j] = x[j - s]
            pm.pts[(g, b)] = enc(p, rot, pt_scale)
    return pm


def rotation_steps(pm: PtMatrix):
    """Rotations (slot steps) the matvec uses."""
    lay = pm.layout
    babies = {b for (_, b) in pm.pts}
    giants = {g for (g, _) in pm.pts}
    return sorted({b for b in babies if b} | {g * lay.n1 for g in giants if g} | set(fold_steps(lay.folds)))


def baby_products(p: ckks.Params, keys: ckks.Keys, pm: PtMatrix, ct: ckks.Ct) -> dict:
    """The first half of the double-hoisted BSGS product: the baby steps in QP
    (one ModUp of c1, no ModDown) and, for every giant step g with diagonals,
    inner_g = sum_b diag'_{g,b} (x) baby_b over the level's QP limbs, as a pair
    of coefficient-domain polynomials.  Returns {g: (inner_g0, inner_g1)}."""
    lay, lvl = pm.layout, ct.level
    if lvl != pm.level:
        raise ValueError("ciphertext level does not match the prepared matrix")
    qp = p.qp_mods(lvl)
    qm = p.q_mods(lvl)
    psis = p.psis(qp)

    # Baby steps in QP, sharing one ModUp of c1 (no ModDown).
    digits = ckks.modup(p, ct.c1, lvl)
    baby = {}
    for b in sorted({b for (_, b) in pm.pts}):
        if b == 0:
            baby[0] = (ckks.lift_times_P(p, ct.c0, lvl), ckks.lift_times_P(p, ct.c1, lvl))
            continue
        k = p.galois(b)
        dr = [ckks.automorphism(p, d, k, qp) for d in digits]
        u0, u1 = ckks.ks_inner(p, dr, ckks._key_for(keys, k), lvl)
        u0 = ring.add(u0, ckks.lift_times_P(p, ckks.automorphism(p, ct.c0, k, qm), lvl), qp)
        baby[b] = (u0, u1)
    # Products are sums of ring products; evaluate them in the oracle's own
    # NTT domain (an exact ring isomorphism) to save transforms, or, with
    # ckks.EXACT, each one by the schoolbook convolution.
    baby_hat = {} if ckks.EXACT else \
        {b: (ring.ntt(u0, qp, psis), ring.ntt(u1, qp, psis)) for b, (u0, u1) in baby.items()}

    inner = {}
    for g in range(lay.n2):
        bs = [b for (gg, b) in pm.pts if gg == g]
        if not bs:
            continue
        s0 = np.zeros((len(qp), p.N), dtype=np.uint64)
        s1 = np.zeros_like(s0)
        for b in bs:
            if ckks.EXACT:
                d = ring.from_signed(pm.pts[(g, b)], qp)
                s0 = ring.add(s0, ckks.polymul(p, d, baby[b][0], qp), qp)
                s1 = ring.add(s1, ckks.polymul(p, d, baby[b][1], qp), qp)
                continue
            dh = ring.ntt(ring.from_signed(pm.pts[(g, b)], qp), qp, psis)
            s0 = ring.add(s0, ring.mul(dh, baby_hat[b][0], qp), qp)
            s1 = ring.add(s1, ring.mul(dh, baby_hat[b][1], qp), qp)
        if ckks.EXACT:
            inner[g] = (s0, s1)
        else:
            inner[g] = (ring.ntt(s0, qp, psis, inverse=True), ring.ntt(s1, qp, psis, inverse=True))
    return inner


def giant_steps(p: ckks.Params, keys: ckks.Keys, pm: PtMatrix, inner: dict, lvl: int, scale: float) -> ckks.Ct:
    """The second half: the giant steps on the QP inner products (for g > 0:
    ModDown the a-part, ModUp, phi, key inner product; the b-part is already
    in QP and only gets phi), one ModDown of the sum, the rescale, then the
    folds.  scale: the product's scale before the rescale."""
    lay = pm.layout
    qp = p.qp_mods(lvl)
    acc0 = np.zeros((len(qp), p.N), dtype=np.uint64)
    acc1 = np.zeros_like(acc0)
    for g in sorted(inner):
        in0, in1 = inner[g]
        if g == 0:
            acc0, acc1 = ring.add(acc0, in0, qp), ring.add(acc1, in1, qp)
            continue
        k = p.galois(g * lay.n1)
        c1q = ckks.moddown(p, in1, lvl)
        dr = [ckks.automorphism(p, d, k, qp) for d in ckks.modup(p, c1q, lvl)]
        k0, k1 = ckks.ks_inner(p, dr, ckks._key_for(keys, k), lvl)
        acc0 = ring.add(acc0, ring.add(ckks.automorphism(p, in0, k, qp), k0, qp), qp)
        acc1 = ring.add(acc1, k1, qp)

    out = ckks.Ct(ckks.moddown(p, acc0, lvl), ckks.moddown(p, acc1, lvl), lvl, scale)
    out = ckks.rescale(p, out)
    out.scale = pm.out_scale
    for stride, radix in lay.folds:
        steps = [d * stride for d in range(1, radix)]
        rots = ckks.rotate_hoisted(p, keys, out, steps)
        acc = out
        for st in steps:
            acc = ckks.add(p, acc, rots[st])
        out = acc
    return out


def matvec(p: ckks.Params, keys: ckks.Keys, pm: PtMatrix, ct: ckks.Ct) -> ckks.Ct:
    """Double-hoisted BSGS y = W x, then rescale, then the folds."""
    return giant_steps(p, keys, pm, baby_products(p, keys, pm, ct), ct.level, ct.scale * pm.pt_scale)


def same_shape(a: PtMatrix, b: PtMatrix) -> bool:
    """Matrices whose products can share their giant steps: the same layout
    (pads, BSGS split, folds), level and scales."""
    return (a.layout == b.layout and a.level == b.level and a.pt_scale == b.pt_scale
            and a.out_scale == b.out_scale)


def matvec_sum(p: ckks.Params, keys: ckks.Keys, pms, cts) -> ckks.Ct:
    """sum_k W_k x_k for matrices of the same shape: the baby-step products
    of every (W_k, x_k) are added in QP, giant step by giant step, and the
    sum goes through one set of giant steps, one ModDown, one rescale and one
    set of folds (reading R31).  All x_k share level and scale."""
    if not pms or len(pms) != len(cts):
        raise ValueError("matvec_sum takes one ciphertext per matrix")
    lvl, scale = cts[0].level, cts[0].scale
    for pm, ct in zip(pms, cts):
        if not same_shape(pm, pms[0]) or ct.level != lvl or ct.scale != scale:
            raise ValueError("matvec_sum: matrices and ciphertexts must share shape, level and scale")
    qp = p.qp_mods(lvl)
    total = {}
    for pm, ct in zip(pms, cts):
        for g, (i0, i1) in baby_products(p, keys, pm, ct).items():
            if g in total:
                total[g] = (ring.add(total[g][0], i0, qp), ring.add(total[g][1], i1, qp))
            else:
                total[g] = (i0, i1)
    return giant_steps(p, keys, pms[0], total, lvl, scale * pms[0].pt_scale)


def matvec_cleartext(W: np.ndarray, x: np.ndarray, in_pad: int, out_pad: int, n: int) -> np.ndarray:
    """What the encrypted matvec must decrypt to, slot by slot (FP64)."""
    xp = np.zeros(in_pad)
    xp[: len(x)] = x
    y = np.zeros(out_pad)
    y[: W.shape[0]] = np.asarray(W, dtype=np.float64) @ xp[: W.shape[1]]
    return y[np.arange(n) % out_pad]
