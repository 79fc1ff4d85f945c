"""HE-LRM: client-side digit selectors, block-diagonal packing, and the
encrypted DLRM pipeline (test infrastructure only).

Paper passages followed:
  - Sec. 3 (private embedding lookup as y = E^T s with a one-hot selector s
    built by the client, evaluated as a plaintext-matrix x ciphertext product
    with the BSGS method, consuming one level);
  - Sec. 4.1 (deterministic base-p digit decomposition, little-endian,
    l = ceil(log_p k); the embedding is sum_j C_j[i_j]);
  - Sec. 4.2.2 (block-diagonal packing of all tables into one matrix, the
    client concatenating the one-hots of all tables into one vector);
  - Sec. 2.2 and Sec. 5.3 (DLRM: bottom MLP, embeddings, interaction, top MLP,
    encrypted logit, sigmoid at the client).

The readings where the paper is silent (activation x^2 everywhere but the last
top layer, the dot-interaction scheme, the level schedule, slot layouts) are
stated at each function.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ckks, linear, poly, ring

DIM = 16


# --------------------------------------------------------------------------
# Client side: digits and selectors (Sec. 4.1, Sec. 4.2.2)
# --------------------------------------------------------------------------
def num_digits(k: int, p: int) -> int:
    """Smallest l >= 1 with p^l >= k (integer loop, no floating-point log)."""
    ell, cap = 1, p
    while cap < k:
        cap *= p
        ell += 1
    return ell


def digits(i: int, p: int, ell: int) -> list:
    """Little-endian base-p digits (i_0, ..., i_{l-1}) of i: i = sum_j i_j p^j."""
    out = []
    for _ in range(ell):
        out.append(i % p)
        i //= p
    return out


def compressed(k: int, p: int, threshold=None) -> bool:
    """Whether a table of k rows is digit-decomposed: k > threshold (Sec. 5.2:
    tables with more rows than a threshold are compressed, base p = 4 there);
    threshold None means p, so a table that fits one digit stays plain."""
    return k > (p if threshold is None else threshold)


def selector_layout(cards, p, threshold=None):
    """[(table, digit, offset, width)]: table t in order, digit j ascending.

    An uncompressed table keeps its plain one-hot of width k; a compressed one
    gets l_t one-hots of width p.
    """
    out, off = [], 0
    for t, k in enumerate(cards):
        if not compressed(k, p, threshold):
            out.append((t, 0, off, k))
            off += k
        else:
            for j in range(num_digits(k, p)):
                out.append((t, j, off, p))
                off += p
    return out, off


def selector_vector(cards, p, indices, threshold=None) -> np.ndarray:
    """The concatenated one-hot digit selectors of one query."""
    lay, width = selector_layout(cards, p, threshold)
    v = np.zeros(width)
    for (t, j, off, w) in lay:
        i = int(indices[t])
        if not compressed(cards[t], p, threshold):
            v[off + i] = 1.0
        else:
            v[off + digits(i, p, num_digits(cards[t], p))[j]] = 1.0
    return v


def replicate(v: np.ndarray, period: int, n: int) -> np.ndarray:
    vp = np.zeros(period)
    vp[: len(v)] = v
    return vp[np.arange(n) % period]


def embedding_matrix(cards, p, tables, row_offset: int, n_rows: int, dim: int = DIM, threshold=None) -> np.ndarray:
    """Block-diagonal packing: table t's transposed compressed tables occupy
    rows [row_offset + dim t, row_offset + dim (t+1)) and the selector columns
    of its digits (torch.block_diag of the per-table [C_0^T ... C_{l-1}^T])."""
    lay, width = selector_layout(cards, p, threshold)
    M = np.zeros((n_rows, width))
    for (t, j, off, w) in lay:
        C = np.asarray(tables[t][j], dtype=np.float64)
        M[row_offset + dim * t: row_offset + dim * (t + 1), off: off + w] = C[:w].T
    return M


# --------------------------------------------------------------------------
# Cleartext FP64 DLRM: the plain definition of the result
# --------------------------------------------------------------------------
def embedding_cleartext(cards, p, tables, indices, threshold=None):
    out = []
    for t, k in enumerate(cards):
        i = int(indices[t])
        if not compressed(k, p, threshold):
            out.append(np.asarray(tables[t][0][i], dtype=np.float64))
        else:
            ds = digits(i, p, num_digits(k, p))
            out.append(sum(np.asarray(tables[t][j][ds[j]], dtype=np.float64) for j in range(len(ds))))
    return out


def activation(spec, v):
    """x^2, or the model's activation polynomial (spec.act, powers of x)."""
    act = getattr(spec, "act", None)
    if act is None:
        return v ** 2
    return np.polynomial.polynomial.polyval(v, np.asarray(act, dtype=np.float64))


def act_const(p: ckks.Params, spec, rows: int, out_pad: int, scale: float):
    """The polynomial's a_0 as a plaintext on the layer's real outputs only
    (rows of each period out_pad), at the activation's output scale: the
    homomorphic polynomial is evaluated without a_0, so the zero padding of
    the layout stays zero (x^2 keeps it zero by itself)."""
    act = getattr(spec, "act", None)
    if act is None or act[0] == 0:
        return None
    return ckks.encode_real(p, replicate(np.full(rows, float(act[0])), out_pad, p.n), scale)


def act_linear(act):
    """The activation polynomial without its constant term (evaluated on the ciphertext)."""
    return (0.0,) + tuple(act[1:])


def activation_levels(spec) -> int:
    """Levels one activation consumes: 1 for x^2, poly.depth(d) for a polynomial."""
    act = getattr(spec, "act", None)
    return 1 if act is None else poly.depth(len(act) - 1)


def dlrm_cleartext(spec, w, dense, indices):
    """Bottom MLP (the activation after every layer), embeddings, interaction
    ([b; e_1..e_T] for concat; [b; <z_a, z_c> for a < c] for dot, pairs in
    lexicographic order), top MLP (the activation after all but the last
    layer); returns (logit, sigmoid(logit), top-MLP input)."""
    h = np.asarray(dense, dtype=np.float64)
    for W, b in zip(w.bottom_W, w.bottom_b):
        h = activation(spec, W @ h + b)
    embs = embedding_cleartext(spec.cards, spec.base, w.tables, indices, spec.threshold)
    blocks = [h] + embs
    if spec.interaction == "dot":
        x = [h] + [np.array([blocks[a] @ blocks[c]]) for a in range(len(blocks))
                   for c in range(a + 1, len(blocks))]
        x = np.concatenate(x)
    else:
        x = np.concatenate(blocks)
    y = x
    for i, (W, b) in enumerate(zip(w.top_W, w.top_b)):
        y = W @ y + b
        if i + 1 < len(w.top_W):
            y = activation(spec, y)
    logit = float(y[0])
    return logit, 1.0 / (1.0 + np.exp(-logit)), x


# --------------------------------------------------------------------------
# Model compilation (layouts, levels, plaintexts)
# --------------------------------------------------------------------------
@dataclass
class Layer:
    pm: linear.PtMatrix
    bias: np.ndarray | None          # signed coefficients at (level - 1), scale = out_scale
    square: bool                     # an activation follows (x^2, or the model's polynomial)
    act_const: np.ndarray | None = None   # polynomial activation: a_0 on the layer's real outputs


@dataclass
class Compiled:
    spec: object
    lvl_dense: int
    lvl_sel: int
    lvl_z: int
    lvl_u: int
    p_dense: int
    p_sel: int
    W_z: int
    W2: int = 0
    W_u: int = 0
    Bp: int = 0                      # blocks in z (with the ones block for dot)
    S: int = 0                       # dot: number of block shifts
    bottom: list = field(default_factory=list)
    emb: linear.PtMatrix | None = None
    # a selector wider than n slots: one matrix per ciphertext (emb is None)
    emb_chunks: list = field(default_factory=list)
    ones: np.ndarray | None = None
    masks: list = field(default_factory=list)       # dot: mask_0 .. mask_S
    mask_scale: float = 0.0
    top: list = field(default_factory=list)
    lvl_h: int = 0                   # level of z = h + e (lvl_z unless z is bootstrapped)
    boots: dict = field(default_factory=dict)       # boot point ("b<i>", "z", "t<i>") -> (boot.Boot, level after)

    def rotation_steps(self):
        st = set()
        for lay in self.bottom + self.top:
            st |= set(linear.rotation_steps(lay.pm))
        for pm in self.emb_pms():
            st |= set(linear.rotation_steps(pm))
        if self.spec.interaction == "dot":
            st.add(-DIM * self.Bp)
            st |= {DIM * s for s in range(1, self.S + 1)}
        for b, _ in self.boots.values():
            st |= set(b.rotation_steps())
        return sorted(st)

    def emb_pms(self):
        return [self.emb] if self.emb is not None else list(self.emb_chunks)

    def n_sel(self) -> int:
        """Ciphertexts of the selector (1 unless it is wider than n slots)."""
        return 1 if self.emb is not None else len(self.emb_chunks)

    def plaintexts(self):
        """Every plaintext of the model, in the canonical order: per bottom
        layer its diagonals in (g, b) order, its bias, then (polynomial
        activation with a_0 != 0) its activation constant; the embedding
        diagonals; (dot) the ones block and the masks 0..S; per top layer the
        same as per bottom layer."""
        def layer(lay):
            return [lay.pm.pts[k] for k in lay.pm.ordered_keys()] + [lay.bias] + \
                ([lay.act_const] if lay.act_const is not None else [])
        out = []
        for lay in self.bottom:
            out += layer(lay)
        for pm in self.emb_pms():
            out += [pm.pts[k] for k in pm.ordered_keys()]
        if self.spec.interaction == "dot":
            out += [self.ones] + list(self.masks)
        for lay in self.top:
            out += layer(lay)
        for name in boot_order(self):
            b = self.boots[name][0]
            for pm in b.cts + [b.stc]:
                out += [pm.pts[k] for k in pm.ordered_keys()]
        return out


def pair_index(a: int, c: int, B: int) -> int:
    """Index of the pair (a, c), a < c < B, in lexicographic order."""
    return sum(B - 1 - x for x in range(a)) + (c - a - 1)


def dot_top_matrix(W0: np.ndarray, B: int, Bp: int, S: int, W2: int, W_u: int) -> np.ndarray:
    """First top layer over the interaction layout: region s-1 (width W2) holds,
    in block a, the products z_a * z_{(a+s) mod B'}; its 16 slots all get the
    weight of pair {a, (a+s) mod B'} (the block sum of the dot product is folded
    into the weights), except pair {0, ones} whose slots carry b_out itself."""
    M = np.zeros((W0.shape[0], W_u))
    for s in range(1, S + 1):
        n_a = Bp // 2 if (Bp % 2 == 0 and s == Bp // 2) else Bp
        for a in range(n_a):
            x, y = sorted((a, (a + s) % Bp))
            cols = (s - 1) * W2 + DIM * a + np.arange(DIM)
            if y == Bp - 1:
                if x == 0:
                    M[:, cols] = W0[:, :DIM]
            else:
                M[:, cols] = W0[:, [DIM + pair_index(x, y, B)]]
    return M


BOOT_POINT_ORDER = "bzt"   # bootstraps run in model order: before bottom layers, on z, before top layers


def boot_order(c) -> list:
    """The model's bootstrap points in the order the inference meets them."""
    def key(name):
        return (BOOT_POINT_ORDER.index(name[0]), int(name[1:]) if name[1:] else 0)
    return sorted(c.boots, key=key)


BOOT_LOG2_BOOST = 8    # activations reach |z| ~ 6: the message is 2^-12 |z| of q_0 in EvalMod


def level_plan(n_bot: int, n_top: int, ad: int, dot: bool, points):
    """Levels as late as possible in every segment between bootstraps (each
    segment ends at level 0, where the next bootstrap or the logit takes it):
    returns {stage: level its input sits at} for the stages "b<i>" (bottom
    layer i), "I" (the interaction on z), "t<i>" (top layer i), and "h" (the
    level of z = h + e).  A bootstrap point "b<i>" (1 <= i < n_bot) runs
    before bottom layer i, "z" before the interaction, "t<i>" (1 <= i < n_top)
    before top layer i.  Costs: a layer 1 + ad (the last top layer 1), the
    dot interaction 2."""
    seq = [(f"b{i}", 1 + ad) for i in range(n_bot)] + [("I", 2 if dot else 0)] + \
        [(f"t{i}", 1 + ad if i + 1 < n_top else 1) for i in range(n_top)]
    cut = {f"b{i}" for i in range(1, n_bot) if f"b{i}" in points} | \
        ({"I"} if "z" in points else set()) | {f"t{i}" for i in range(1, n_top) if f"t{i}" in points}
    bad = set(points) - {f"b{i}" for i in range(1, n_bot)} - {"z"} - {f"t{i}" for i in range(1, n_top)}
    if bad:
        raise ValueError(f"unknown bootstrap points {sorted(bad)}")
    lv, out = 0, {}
    for name, cost in reversed(seq):
        lv += cost
        out[name] = lv
        if name in cut:
            lv = 0
    out["h"] = out["I"] if "z" not in points else 0
    return out


def compile_model(p: ckks.Params, spec, w) -> Compiled:
    """Levels are assigned as late as possible so the logit ends at level 0:
    each matvec consumes one level, each activation one (x^2) or poly.depth(d)
    (a degree-d polynomial), the dot interaction two.  With bootstrap points
    (spec.boot) every segment between them is planned the same way and ends
    at level 0, and a bootstrap (boot.bootstrap, 512 or fewer periodic slots)
    lifts the ciphertext to the next segment's first level."""
    T = len(spec.cards)
    B = T + 1
    n_bot, n_top = len(w.bottom_W), len(w.top_W)
    act = getattr(spec, "act", None)
    ad = activation_levels(spec)
    dot = spec.interaction == "dot"
    points = tuple(getattr(spec, "boot", ()) or ())
    plan = level_plan(n_bot, n_top, ad, dot, points)
    lvl_u = plan["t0"]
    lvl_z = plan["I"]
    lvl_h = plan["h"]
    lvl_sel = lvl_h + 1
    lvl_dense = plan["b0"]
    cap = p.L
    if points:
        from . import boot as _boot
        cap = p.L - _boot.levels_used(_boot.BootParams(n_s=1))
    need = max(v for k, v in plan.items() if k != "h")
    if need > cap or lvl_sel > cap:
        raise ValueError(f"model needs {max(need, lvl_sel)} levels, chain has {cap}")
    Bp = B + 1 if dot else B
    W_z = linear.pow2ceil(DIM * Bp)
    lay_sel, sel_w = selector_layout(spec.cards, spec.base, spec.threshold)
    c = Compiled(spec, lvl_dense, lvl_sel, lvl_z, lvl_u, linear.pow2ceil(spec.n_dense),
                 min(linear.pow2ceil(sel_w), p.n), W_z, Bp=Bp, lvl_h=lvl_h)

    def bootstrap_point(name, period, lvl_now, scale_now, lvl_next):
        """A bootstrap at `name` of a ciphertext at level 0 with `period`-periodic slots."""
        from . import boot as _boot
        assert lvl_now == 0
        bt = _boot.prepare(p, _boot.BootParams(n_s=period, log2_boost=BOOT_LOG2_BOOST, s_ref=scale_now,
                                               coeffs=getattr(spec, "boot_coeffs", None)))
        c.boots[name] = (bt, lvl_next)
        return lvl_next, _boot.out_scale(p, bt, scale_now)
    if dot:
        c.W2 = linear.pow2ceil(2 * DIM * Bp)
        c.S = Bp // 2
        c.W_u = linear.pow2ceil(c.S * c.W2)
    else:
        c.W_u = W_z
    if max(c.W_u, c.p_sel, W_z) > p.n:
        raise ValueError("layout wider than the slot count")

    delta = p.delta
    # Bottom MLP
    lvl, scale, in_pad = lvl_dense, delta, c.p_dense
    for i, (W, b) in enumerate(zip(w.bottom_W, w.bottom_b)):
        last = i + 1 == n_bot
        if f"b{i}" in points and i > 0:
            lvl, scale = bootstrap_point(f"b{i}", in_pad, lvl, scale, plan[f"b{i}"])
        out_pad = W_z if last else linear.pow2ceil(W.shape[0])
        pm = linear.prepare(p, W, in_pad, out_pad, lvl, scale, delta)
        bias = ckks.encode_real(p, replicate(b, out_pad, p.n), delta)
        c.bottom.append(Layer(pm, bias, True))
        lvl -= 1
        if act is None:
            scale = (delta * delta) / p.q[lvl]
            lvl -= 1
        else:
            lvl, scale = poly.simulate(p.q, lvl, delta, act_linear(act), delta)
            c.bottom[-1].act_const = act_const(p, spec, W.shape[0], out_pad, scale)
        in_pad = out_pad
    assert lvl == lvl_h
    scale_b = scale
    # Embedding lookup (block-diagonal, rows [16, 16 (T+1)) of the z layout)
    M = embedding_matrix(spec.cards, spec.base, w.tables, DIM, DIM * B, threshold=spec.threshold)
    if sel_w <= p.n:
        c.emb = linear.prepare(p, M, c.p_sel, W_z, lvl_sel, delta, scale_b)
    else:
        c.emb_chunks = prepare_multi(p, M, W_z, lvl_sel, delta, scale_b)
    scale_z = scale_b
    if "z" in points:
        _, scale_z = bootstrap_point("z", W_z, lvl_h, scale_b, lvl_z)
    if dot:
        ones = np.zeros(W_z)
        ones[DIM * B: DIM * B + DIM] = 1.0
        c.ones = ckks.encode_real(p, replicate(ones, W_z, p.n), scale_b)
        c.mask_scale = float(p.q[lvl_z]) * delta / scale_z
        j = np.arange(p.n)
        c.masks.append(ckks.encode_real(p, ((j % c.W2) < DIM * Bp).astype(float), c.mask_scale))
        for s in range(1, c.S + 1):
            n_a = Bp // 2 if (Bp % 2 == 0 and s == Bp // 2) else Bp
            lo = (s - 1) * c.W2
            m = (((j % c.W_u) >= lo) & ((j % c.W_u) < lo + DIM * n_a)).astype(float)
            c.masks.append(ckks.encode_real(p, m, c.mask_scale))
        u_scale = (delta * delta) / p.q[lvl_z - 1]
    else:
        u_scale = scale_z
    # Top MLP
    lvl, scale = lvl_u, u_scale
    for i, (W, b) in enumerate(zip(w.top_W, w.top_b)):
        last = i + 1 == n_top
        if f"t{i}" in points and i > 0:
            lvl, scale = bootstrap_point(f"t{i}", linear.pow2ceil(w.top_W[i - 1].shape[0]), lvl, scale,
                                         plan[f"t{i}"])
        if i == 0:
            in_pad = c.W_u
            Wm = dot_top_matrix(W, B, Bp, c.S, c.W2, c.W_u) if dot else W
        else:
            in_pad = linear.pow2ceil(W.shape[1])
            Wm = W
        out_pad = linear.pow2ceil(W.shape[0])
        pm = linear.prepare(p, Wm, in_pad, out_pad, lvl, scale, delta)
        bias = ckks.encode_real(p, replicate(b, out_pad, p.n), delta)
        c.top.append(Layer(pm, bias, not last))
        lvl -= 1
        scale = delta
        if not last:
            if act is None:
                scale = (delta * delta) / p.q[lvl]
                lvl -= 1
            else:
                lvl, scale = poly.simulate(p.q, lvl, delta, act_linear(act), delta)
                c.top[-1].act_const = act_const(p, spec, W.shape[0], out_pad, scale)
    assert lvl == 0
    return c


# --------------------------------------------------------------------------
# The encrypted pipeline (Sec. 5.3)
# --------------------------------------------------------------------------
def query_slots(p: ckks.Params, c: Compiled, dense, indices):
    """Client packing: dense features with period p_dense; concatenated digit
    one-hots with period p_sel (a list of per-ciphertext slot vectors when the
    selector is wider than n slots)."""
    xd = replicate(np.asarray(dense, dtype=np.float64), c.p_dense, p.n)
    sel = selector_vector(c.spec.cards, c.spec.base, indices, c.spec.threshold)
    if c.emb is None:
        return xd, chunk_slots(sel, p.n)
    return xd, replicate(sel, c.p_sel, p.n)


def encrypt_query(p, keys, c: Compiled, dense, indices, seed: int):
    """ct_dense with `seed` at lvl_dense, ct_sel with `seed + 1` at lvl_sel, both at
    Delta; a selector of several ciphertexts uses seeds seed + 1, seed + 2, ..."""
    xd, xs = query_slots(p, c, dense, indices)
    ct_d = ckks.encrypt(p, keys, ckks.encode_real(p, xd, p.delta), c.lvl_dense, p.delta, seed)
    if c.emb is None:
        return ct_d, [ckks.encrypt(p, keys, ckks.encode_real(p, x, p.delta), c.lvl_sel, p.delta, seed + 1 + k)
                      for k, x in enumerate(xs)]
    ct_s = ckks.encrypt(p, keys, ckks.encode_real(p, xs, p.delta), c.lvl_sel, p.delta, seed + 1)
    return ct_d, ct_s


def _dense_layer(p, keys, lay: Layer, x: ckks.Ct, act=None) -> ckks.Ct:
    y = linear.matvec(p, keys, lay.pm, x)
    y = ckks.add_pt(p, y, lay.bias, y.scale)
    if lay.square:
        if act is None:
            y = ckks.square(p, keys, y)
        else:   # the polynomial without a_0, then a_0 on the real outputs only
            y = poly.poly_eval(p, keys, y, act_linear(act), p.delta)
            if lay.act_const is not None:
                y = ckks.add_pt(p, y, lay.act_const, y.scale)
    return y


def dot_interaction(p, keys, c: Compiled, z: ckks.Ct) -> ckks.Ct:
    """Pairwise products of the z blocks in two levels.

    z1 = z masked to one period of W2 (first 16 B' slots); zz = z1 + rot(z1,
    -16 B') repeats the blocks so block a+s reads z_{(a+s) mod B'}; A_s = z
    masked to region s-1 of the W_u layout; u = relin(sum_s A_s (x) rot(zz, 16 s))
    rescaled: region s-1, block a holds z_a * z_{(a+s) mod B'}.
    """
    z1 = ckks.rescale(p, ckks.mul_pt(p, z, c.masks[0], c.mask_scale))
    z1.scale = p.delta
    A = []
    for s in range(1, c.S + 1):
        a = ckks.rescale(p, ckks.mul_pt(p, z, c.masks[s], c.mask_scale))
        a.scale = p.delta
        A.append(a)
    zz = ckks.add(p, z1, ckks.rotate(p, keys, z1, -DIM * c.Bp))
    R = ckks.rotate_hoisted(p, keys, zz, [DIM * s for s in range(1, c.S + 1)])
    lvl = z1.level
    mods = p.q_mods(lvl)
    acc = None
    for s in range(1, c.S + 1):
        d = ckks.tensor(p, A[s - 1], R[DIM * s])
        acc = d if acc is None else tuple(ring.add(x, y, mods) for x, y in zip(acc, d))
    return ckks.rescale(p, ckks.relinearize(p, keys, acc, lvl, p.delta * p.delta))


def infer_stages(p, keys, c: Compiled, ct_dense: ckks.Ct, ct_sel):
    """The steps of infer(), in order, as callables that each run one stage
    (a bottom layer; the lookup and z = h + e; the interaction; a top layer)
    on a shared state; after the last one state["y"] is the logit
    ciphertext.  ct_sel: one ciphertext, or the list of them for a selector
    wider than n slots."""
    st = {"h": ct_dense}
    act = getattr(c.spec, "act", None)

    def boot_at(name, x):
        if name not in c.boots:
            return x
        from . import boot as _boot
        bt, lvl_next = c.boots[name]
        return ckks.drop_level(p, _boot.bootstrap(p, keys, bt, x), lvl_next)

    def bottom(i, lay):
        st["h"] = _dense_layer(p, keys, lay, boot_at(f"b{i}", st["h"]), act)

    def lookup():
        e = lookup_multi(p, keys, c.emb_chunks, ct_sel) if c.emb is None else linear.matvec(p, keys, c.emb, ct_sel)
        st["y"] = ckks.add(p, st["h"], e)

    def interaction():
        z = st["y"]
        if c.spec.interaction == "dot":
            z = ckks.add_pt(p, z, c.ones, z.scale)
            st["y"] = dot_interaction(p, keys, c, boot_at("z", z))
        else:
            st["y"] = boot_at("z", z)

    def top(i, lay):
        st["y"] = _dense_layer(p, keys, lay, boot_at(f"t{i}", st["y"]), act)

    stages = [lambda i=i, lay=lay: bottom(i, lay) for i, lay in enumerate(c.bottom)] + [lookup, interaction] + \
        [lambda i=i, lay=lay: top(i, lay) for i, lay in enumerate(c.top)]
    return stages, st


def infer(p, keys, c: Compiled, ct_dense: ckks.Ct, ct_sel) -> ckks.Ct:
    """ct_sel: one ciphertext, or the list of them for a selector wider than n slots."""
    stages, st = infer_stages(p, keys, c, ct_dense, ct_sel)
    for f in stages:
        f()
    return st["y"]


def decrypt_logit(p, sk, ct: ckks.Ct):
    logit = float(ckks.decrypt(p, sk, ct, 1)[0])
    return logit, 1.0 / (1.0 + np.exp(-logit))


# --------------------------------------------------------------------------
# The stand-alone lookup (the tiny workload): one table, digits in base p
# --------------------------------------------------------------------------
def lookup_matrix(tables, p_base: int, k: int) -> np.ndarray:
    """dim x (l p) matrix [C_0^T ... C_{l-1}^T] of one compressed table."""
    return embedding_matrix([k], p_base, [tables], 0, DIM)


# --------------------------------------------------------------------------
# Selectors wider than the slot count (Sec. 3.2.1 and Sec. 5.4: a client's
# one-hot vector of k_t entries needs ceil(k_t / n) ciphertexts; the paper's
# least-compressed Criteo models take 18 and 85 input ciphertexts, and the
# lookup with two input ciphertexts has 1024 non-zero diagonals)
# --------------------------------------------------------------------------
def selector_chunks(width: int, n: int):
    """[(first column, columns)] of the ceil(width / n) ciphertexts: chunk c
    holds selector columns [c n, min((c + 1) n, width))."""
    return [(c0, min(n, width - c0)) for c0 in range(0, width, n)]


def prepare_multi(p: ckks.Params, M: np.ndarray, out_pad: int, level: int, ct_scale: float,
                  target_scale: float):
    """One BSGS matrix per chunk: the columns of M that chunk c holds, padded
    to in_pad_c = pow2ceil(columns) (so all but the last chunk have in_pad = n)."""
    out = []
    for c0, w in selector_chunks(M.shape[1], p.n):
        out.append(linear.prepare(p, M[:, c0:c0 + w], linear.pow2ceil(w), out_pad, level, ct_scale, target_scale))
    return out


def chunk_slots(sel: np.ndarray, n: int):
    """The slots of each chunk's ciphertext: its columns replicated with its period."""
    return [replicate(sel[c0:c0 + w], linear.pow2ceil(w), n) for c0, w in selector_chunks(len(sel), n)]


def lookup_groups(pms):
    """The chunks' matrices grouped by shape (linear.same_shape), in order of
    first appearance: [[chunk indices], ...].  All but the last chunk hold n
    columns, so there are at most two groups."""
    groups = []
    for k, pm in enumerate(pms):
        for grp in groups:
            if linear.same_shape(pms[grp[0]], pm):
                grp.append(k)
                break
        else:
            groups.append([k])
    return groups


def lookup_multi(p: ckks.Params, keys: ckks.Keys, pms, cts):
    """y = M s = sum_c M_c s_c.  The chunks of one shape share their giant
    steps, ModDown, rescale and folds (linear.matvec_sum, reading R31); the
    groups' results are added in order."""
    out = None
    for grp in lookup_groups(pms):
        y = linear.matvec_sum(p, keys, [pms[k] for k in grp], [cts[k] for k in grp])
        out = y if out is None else ckks.add(p, out, y)
    return out
