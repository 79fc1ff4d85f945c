// dlrm.cu -- HE-LRM on top of the CKKS layer.
//
//  * client: base-p digits of each index (little-endian, l = ceil(log_p k),
//    Sec. 4.1), one one-hot per digit, all tables' selectors concatenated
//    (Sec. 4.2.2), replicated with the selector's period, encoded, encrypted;
//  * server: block-diagonal packing of every table's transposed compressed
//    tables into one matrix, so the lookup of all tables is one BSGS matvec
//    that consumes one level and leaves the embeddings contiguous (Sec. 4.2);
//  * DLRM (Sec. 2.2, Sec. 5.3): bottom MLP, embeddings, interaction, top MLP,
//    encrypted logit; x^2 activations after every layer but the last.
//
// Model layout (the reading used by library and oracle alike): z holds
// blocks of 16 slots with period W_z = pow2ceil(16 B'): block 0 = bottom MLP
// output, block t = embedding of table t-1, and for the dot interaction a block
// of ones (B' = T + 2).  Dot interaction in two levels: z1 = z masked to the
// first 16 B' slots of each period W2 = pow2ceil(32 B'); zz = z1 + rot(z1, -16 B')
// repeats the blocks; A_s = z masked to region s-1 of the top-input layout
// (period W_u); u = relin(sum_s A_s (x) rot(zz, 16 s)), s = 1..B'/2, so region
// s-1, block a holds z_a * z_{(a+s) mod B'}; the first top layer sums the 16
// slots of each pair in its weights.  Levels are assigned as late as possible so
// the logit ends at level 0.  The layers are evaluated by batch.cu (one query
// is a batch of one).
#include <algorithm>
#include <cmath>

#include "model.cuh"

namespace helrm {



static int num_digits(u64 k, u64 p)
{
    int ell = 1;
    unsigned __int128 cap = p;
    while (cap < k) {
        cap *= p;
        ell++;
    }
    return ell;
}

// Sec. 5.2: a table is digit-decomposed (base p) only if it has more rows than
// the threshold; otherwise it keeps its plain one-hot (threshold p: a table
// that fits one digit).
static bool compressed(u64 k, int p, u64 threshold) { return k > threshold; }

static std::vector<SelSeg> selector_layout(const std::vector<u64> &cards, int p, u64 threshold, int *width)
{
    std::vector<SelSeg> out;
    long off = 0;
    for (int t = 0; t < (int)cards.size(); t++) {
        HCHECK(compressed(cards[t], p, threshold) || cards[t] <= (u64)1 << 30, HELRM_E_PARAM,
               "uncompressed table too large for one selector");
        if (!compressed(cards[t], p, threshold)) {
            out.push_back({t, 0, (int)off, (int)cards[t]});
            off += (long)cards[t];
        } else {
            int ell = num_digits(cards[t], p);
            for (int j = 0; j < ell; j++) {
                out.push_back({t, j, (int)off, p});
                off += p;
            }
        }
        HCHECK(off < (1L << 30), HELRM_E_PARAM, "selector wider than 2^30 slots");
    }
    *width = (int)off;
    return out;
}


// Columns [c0, c0 + w) of the packed lookup matrix: rows [out_offset + dim t,
// out_offset + dim (t+1)) take table t's transposed digit tables at the
// selector columns of its digits.
static std::vector<double> emb_matrix(const Emb &e, const float *const *tables, int out_offset, int rows, int c0,
                                      int w)
{
    std::vector<double> M((size_t)rows * w, 0.0);
    std::vector<int> row0(e.cards.size(), 0);
    for (auto &s : e.layout) {
        const float *C = tables[s.t] + (size_t)row0[s.t] * e.dim;
        for (int r = 0; r < s.width; r++) {
            const int col = s.off + r - c0;
            if (col < 0 || col >= w) continue;
            for (int kk = 0; kk < e.dim; kk++)
                M[(size_t)(out_offset + e.dim * s.t + kk) * w + col] = (double)C[(size_t)r * e.dim + kk];
        }
        row0[s.t] += s.width;
    }
    return M;
}

Emb *emb_prepare(Ctx *c, const std::vector<u64> &cards, int base, u64 threshold, int dim, const float *const *tables,
                 int out_offset, int out_pad, int level, double ct_scale, double target_scale)
{
    HCHECK(!cards.empty() && base >= 2 && dim >= 1 && tables, HELRM_E_INVAL, "bad embedding description");
    for (u64 k2 : cards) HCHECK(k2 >= 1, HELRM_E_INVAL, "table with no rows");
    std::unique_ptr<Emb> e(new Emb(c));
    e->cards = cards;
    e->base = base;
    e->threshold = threshold ? threshold : (u64)base;
    e->dim = dim;
    e->layout = selector_layout(cards, base, e->threshold, &e->width);
    e->in_pad = pow2ceil(e->width);
    e->out_pad = out_pad;
    const int rows = out_offset + dim * (int)cards.size();
    HCHECK(rows <= out_pad, HELRM_E_INVAL, "embedding outputs exceed out_pad");
    if (e->in_pad <= c->n_slots) {
        std::vector<double> M = emb_matrix(*e, tables, out_offset, rows, 0, e->width);
        e->pm.reset(ptmat_prepare(c, M.data(), rows, e->width, e->in_pad, out_pad, level, ct_scale, target_scale));
    } else {   // one matrix per ciphertext of the selector
        e->in_pad = c->n_slots;
        for (int c0 = 0; c0 < e->width; c0 += c->n_slots) {
            const int w = std::min(c->n_slots, e->width - c0);
            std::vector<double> M = emb_matrix(*e, tables, out_offset, rows, c0, w);
            e->chunks.emplace_back(
                ptmat_prepare(c, M.data(), rows, w, pow2ceil(w), out_pad, level, ct_scale, target_scale));
        }
    }
    std::vector<int> tab;
    for (size_t t = 0; t < cards.size(); t++) {
        int off = -1;
        for (auto &s : e->layout)
            if (s.t == (int)t) {
                off = s.off;
                break;
            }
        tab.push_back((int)std::min<u64>(cards[t], (u64)1 << 30));
        tab.push_back(off);
        // digits of a compressed table; 0 = a plain one-hot of `rows` slots
        tab.push_back(compressed(cards[t], base, e->threshold) ? num_digits(cards[t], base) : 0);
    }
    e->d_tab = DevMem(c, tab.size() * 4);
    CUDA_CHECK(cudaMemcpyAsync(e->d_tab.ptr, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    return e.release();
}

void emb_pack_host(const Emb *e, const u64 *indices, std::vector<double> &sel)
{
    sel.assign(e->width, 0.0);
    for (auto &s : e->layout) {
        u64 i = indices[s.t];
        HCHECK(i < e->cards[s.t], HELRM_E_INVAL, "index out of range for its table");
        if (!compressed(e->cards[s.t], e->base, e->threshold)) {
            sel[s.off + i] = 1.0;
        } else {
            for (int j = 0; j < s.j; j++) i /= (u64)e->base;
            sel[s.off + (int)(i % (u64)e->base)] = 1.0;
        }
    }
}

// ------------------------------------------------------------------ model


static int pair_index(int a, int c2, int B)
{
    int idx = 0;
    for (int x = 0; x < a; x++) idx += B - 1 - x;
    return idx + (c2 - a - 1);
}

static Plaintext *encode_vec(Ctx *c, const std::vector<double> &v, int level, double scale, int form)
{
    return pt_encode(c, v.data(), (int)v.size(), (int)v.size(), level, false, scale, form);
}

static std::vector<double> replicate_bias(const double *b, int n, int period)
{
    std::vector<double> v(period, 0.0);
    for (int i = 0; i < n; i++) v[i] = b[i];
    return v;
}

Model *model_create(Ctx *c, const helrm_model_desc *d)
{
    HCHECK(d && d->dim == DIM, HELRM_E_INVAL, "model dim must be 16");
    HCHECK(d->n_bottom >= 1 && d->n_top >= 1 && d->n_tables >= 1, HELRM_E_INVAL, "empty model");
    HCHECK(d->bottom_widths[0] == d->n_dense && d->bottom_widths[d->n_bottom] == DIM, HELRM_E_INVAL,
           "bottom MLP must map n_dense -> 16");
    HCHECK(d->top_widths[d->n_top] == 1, HELRM_E_INVAL, "top MLP must end in one logit");
    HCHECK(d->interaction == 0 || d->interaction == 1, HELRM_E_INVAL, "interaction must be 0 (dot) or 1 (concat)");
    std::unique_ptr<Model> m(new Model(c));
    const bool dot = d->interaction == 0;
    m->n_dense = (int)d->n_dense;
    m->interaction = d->interaction;
    m->T = (int)d->n_tables;
    m->B = m->T + 1;
    const int nb = (int)d->n_bottom, nt = (int)d->n_top;
    const u32 want_top = dot ? DIM + m->B * (m->B - 1) / 2 : DIM * m->B;
    HCHECK(d->top_widths[0] == want_top, HELRM_E_INVAL, "top MLP input width does not match the interaction");
    // the activation: x^2 (one level) or a polynomial (poly_depth(d) levels),
    // evaluated without its a_0, which is added on the real outputs only
    std::vector<double> act, act_lin;
    if (d->act_degree) {
        HCHECK(d->act_coeffs, HELRM_E_INVAL, "act_coeffs is NULL");
        act.assign(d->act_coeffs, d->act_coeffs + d->act_degree + 1);
        act_lin = act;
        act_lin[0] = 0.0;
    }
    const int ad = act.empty() ? 1 : poly_depth((int)d->act_degree);
    // Bootstrap points split the network into segments; every segment is
    // planned as late as possible and ends at level 0 (costs: a layer 1 + ad,
    // the last top layer 1, the dot interaction 2).
    HCHECK((d->boot_bottom & 1u) == 0 && (d->boot_top & 1u) == 0 && (nb >= 32 || (d->boot_bottom >> nb) == 0) &&
               (nt >= 32 || (d->boot_top >> nt) == 0),
           HELRM_E_INVAL, "bootstrap points must lie before bottom / top layers 1 .. n-1");
    std::vector<char> pb(nb, 0), pt(nt, 0);
    for (int i = 1; i < nb; i++) pb[i] = (d->boot_bottom >> i) & 1u;
    for (int i = 1; i < nt; i++) pt[i] = (d->boot_top >> i) & 1u;
    const bool pz = d->boot_z != 0;
    std::vector<int> lv_b(nb), lv_t(nt);
    int lv = 0;
    for (int i = nt - 1; i >= 0; i--) {
        lv += (i + 1 < nt) ? 1 + ad : 1;
        lv_t[i] = lv;
        if (pt[i]) lv = 0;
    }
    lv += dot ? 2 : 0;
    const int lv_I = lv;
    if (pz) lv = 0;
    for (int i = nb - 1; i >= 0; i--) {
        lv += 1 + ad;
        lv_b[i] = lv;
        if (pb[i]) lv = 0;
    }
    const bool boots = pz || std::count(pb.begin(), pb.end(), 1) || std::count(pt.begin(), pt.end(), 1);
    const int boot_levels = 1 + poly_depth(16) + 6 + 1;   // the bootstraps' CoeffToSlot, cosine, double angles, SlotToCoeff
    const int cap = boots ? c->L - boot_levels : c->L;
    m->lvl_u = lv_t[0];
    m->lvl_z = lv_I;
    m->lvl_h = pz ? 0 : lv_I;
    m->lvl_sel = m->lvl_h + 1;
    m->lvl_dense = lv_b[0];
    int need = std::max({*std::max_element(lv_b.begin(), lv_b.end()), *std::max_element(lv_t.begin(), lv_t.end()),
                         lv_I, m->lvl_sel});
    HCHECK(need <= cap, HELRM_E_PARAM,
           "model needs " + std::to_string(need) + " levels, chain has " + std::to_string(cap) +
               (boots ? " below its bootstrapping levels" : ""));
    m->boot_b.resize(nb);
    m->boot_t.resize(nt);
    std::vector<double> boot_coeffs;
    if (d->boot_coeffs) boot_coeffs.assign(d->boot_coeffs, d->boot_coeffs + 17);
    // a bootstrap of the level-0 ciphertext with period-n_s slots and scale `scale`
    auto boot_point = [&](Model::BootPoint &bp, int n_s, int &lvl, double &scale, int lvl_next) {
        HCHECK(lvl == 0, HELRM_E_PARAM, "internal: a segment does not end at level 0");
        BootDesc bd{n_s, 24, 6, 16, 8, 1, scale, std::ldexp(1.0, 60), boot_coeffs};
        bp.b.reset(boot_create(c, bd));
        bp.lvl_next = lvl_next;
        scale = bp.b->out_scale(scale);
        lvl = lvl_next;
    };
    m->Bp = dot ? m->B + 1 : m->B;
    m->W_z = pow2ceil(DIM * m->Bp);
    m->p_dense = pow2ceil(m->n_dense);
    if (dot) {
        m->W2 = pow2ceil(2 * DIM * m->Bp);
        m->S = m->Bp / 2;
        m->W_u = pow2ceil(m->S * m->W2);
    } else {
        m->W_u = m->W_z;
    }
    int width = 0;
    std::vector<u64> cards(d->cards, d->cards + d->n_tables);
    const u64 thr = d->threshold ? d->threshold : (u64)d->base_p;
    selector_layout(cards, (int)d->base_p, thr, &width);
    // (a selector wider than n slots spans several ciphertexts)
    HCHECK(std::max({m->W_u, m->W_z, m->p_dense}) <= c->n_slots, HELRM_E_PARAM, "layout wider than the slot count");

    const double delta = c->delta;
    // after a layer's matvec (and bias) at level lvl: the activation's level and scale
    auto activate = [&](Layer &L, int rows, int out_pad, int &lvl, double &scale) {
        if (act.empty()) {
            scale = (delta * delta) / (double)c->primes[lvl];
            lvl -= 1;
            return;
        }
        L.act.reset(act_plan(c, act_lin, lvl, delta, delta));
        lvl = L.act->out_level;
        scale = L.act->out_scale;
        if (act[0] != 0.0) {
            std::vector<double> a0(rows, act[0]);
            L.act_const.reset(encode_vec(c, replicate_bias(a0.data(), rows, out_pad), lvl, scale, PT_PLAIN));
        }
    };
    int lvl = m->lvl_dense, in_pad = m->p_dense;
    double scale = delta;
    for (int i = 0; i < nb; i++) {
        const int rows = (int)d->bottom_widths[i + 1], cols = (int)d->bottom_widths[i];
        const int out_pad = (i + 1 == nb) ? m->W_z : pow2ceil(rows);
        if (pb[i]) boot_point(m->boot_b[i], in_pad, lvl, scale, lv_b[i]);
        Layer L;
        L.pm.reset(ptmat_prepare(c, d->bottom_W[i], rows, cols, in_pad, out_pad, lvl, scale, delta));
        L.bias.reset(encode_vec(c, replicate_bias(d->bottom_b[i], rows, out_pad), lvl - 1, delta, PT_PLAIN));
        L.square = true;
        lvl -= 1;
        activate(L, rows, out_pad, lvl, scale);
        m->bottom.push_back(std::move(L));
        in_pad = out_pad;
    }
    HCHECK(lvl == m->lvl_h, HELRM_E_PARAM, "internal: the bottom MLP does not end at the lookup's level");
    const double scale_b = scale;
    m->emb.reset(emb_prepare(c, cards, (int)d->base_p, thr, DIM, d->tables, DIM, m->W_z, m->lvl_sel, delta, scale_b));
    double scale_z = scale_b;
    if (pz) boot_point(m->boot_z, m->W_z, lvl, scale_z, lv_I);
    double u_scale = scale_z;
    if (dot) {
        std::vector<double> ones(m->W_z, 0.0);
        for (int kk = 0; kk < DIM; kk++) ones[DIM * m->B + kk] = 1.0;
        m->ones.reset(encode_vec(c, ones, m->lvl_h, scale_b, PT_PLAIN));
        m->mask_scale = (double)c->primes[m->lvl_z] * delta / scale_z;
        std::vector<double> m0(m->W2, 0.0);
        for (int j = 0; j < DIM * m->Bp; j++) m0[j] = 1.0;
        m->masks.emplace_back(encode_vec(c, m0, m->lvl_z, m->mask_scale, PT_MONT));
        for (int s = 1; s <= m->S; s++) {
            const int n_a = (m->Bp % 2 == 0 && s == m->Bp / 2) ? m->Bp / 2 : m->Bp;
            std::vector<double> ms(m->W_u, 0.0);
            for (int j = 0; j < DIM * n_a; j++) ms[(size_t)(s - 1) * m->W2 + j] = 1.0;
            m->masks.emplace_back(encode_vec(c, ms, m->lvl_z, m->mask_scale, PT_MONT));
        }
        u_scale = (delta * delta) / (double)c->primes[m->lvl_z - 1];
    }
    lvl = m->lvl_u;
    scale = u_scale;
    for (int i = 0; i < nt; i++) {
        const bool last = i + 1 == nt;
        const int rows = (int)d->top_widths[i + 1], cols = (int)d->top_widths[i];
        const int out_pad = pow2ceil(rows);
        if (pt[i]) boot_point(m->boot_t[i], pow2ceil(cols), lvl, scale, lv_t[i]);
        Layer L;
        if (i == 0 && dot) {
            // first top layer over the interaction layout
            std::vector<double> Wm((size_t)rows * m->W_u, 0.0);
            const double *W0 = d->top_W[0];
            for (int s = 1; s <= m->S; s++) {
                const int n_a = (m->Bp % 2 == 0 && s == m->Bp / 2) ? m->Bp / 2 : m->Bp;
                for (int a = 0; a < n_a; a++) {
                    int x = a, y = (a + s) % m->Bp;
                    if (x > y) std::swap(x, y);
                    for (int kk = 0; kk < DIM; kk++) {
                        const size_t col = (size_t)(s - 1) * m->W2 + DIM * a + kk;
                        for (int r = 0; r < rows; r++) {
                            double w = 0.0;
                            if (y == m->Bp - 1) {
                                if (x == 0) w = W0[(size_t)r * cols + kk];
                            } else {
                                w = W0[(size_t)r * cols + DIM + pair_index(x, y, m->B)];
                            }
                            Wm[(size_t)r * m->W_u + col] = w;
                        }
                    }
                }
            }
            L.pm.reset(ptmat_prepare(c, Wm.data(), rows, m->W_u, m->W_u, out_pad, lvl, scale, delta));
        } else {
            const int ip = (i == 0) ? m->W_u : pow2ceil(cols);
            L.pm.reset(ptmat_prepare(c, d->top_W[i], rows, cols, ip, out_pad, lvl, scale, delta));
        }
        L.bias.reset(encode_vec(c, replicate_bias(d->top_b[i], rows, out_pad), lvl - 1, delta, PT_PLAIN));
        L.square = !last;
        lvl -= 1;
        scale = delta;
        if (!last) activate(L, rows, out_pad, lvl, scale);
        m->top.push_back(std::move(L));
    }
    HCHECK(lvl == 0, HELRM_E_PARAM, "internal: level schedule does not end at 0");
    m->act = act;
    c->check_device_errors();
    return m.release();
}

void model_import(Ctx *c, Model *m, const i64 *coeffs, u32 count)
{
    auto pts = m->plaintexts();
    HCHECK(count == pts.size(), HELRM_E_INVAL,
           "plaintext count mismatch: model has " + std::to_string(pts.size()));
    for (size_t i = 0; i < pts.size(); i++) {
        Plaintext *o = pts[i]->get();
        pts[i]->reset(pt_from_signed(c, coeffs + i * (size_t)c->N, o->level, o->qp, o->scale, o->form));
    }
    for (auto &l : m->bottom) l.pm->upload_index();
    if (m->emb->pm) m->emb->pm->upload_index();
    for (auto &ch : m->emb->chunks) ch->upload_index();
    for (auto &l : m->top) l.pm->upload_index();
    for (const Model::BootPoint *bp : m->boot_points())
        for (PtMatrix *pm : bp->b->matrices()) pm->upload_index();
}

void model_export(Ctx *c, Model *m, i64 *coeffs, u32 count)
{
    auto pts = m->plaintexts();
    HCHECK(count == pts.size(), HELRM_E_INVAL, "plaintext count mismatch");
    for (size_t i = 0; i < pts.size(); i++) pt_export_signed(c, pts[i]->get(), coeffs + i * (size_t)c->N);
}

struct Batch;
Batch *batch_create(Ctx *c, const Model *m, const std::vector<const EvalKey *> &evk);
void batch_destroy(Batch *b);
std::vector<Ciphertext *> model_infer_batch(Ctx *c, const Batch *bt, const std::vector<const Ciphertext *> &ct_dense,
                                            const std::vector<const Ciphertext *> &ct_sel);

// One query runs as a batch of one (batch.cu): the same integer operations
// as the op-by-op path below, with the independent steps of each layer (all
// giant steps, all masks, all rotations of the interaction) merged into one
// launch each.
Ciphertext *model_infer(Ctx *c, const EvalKey *evk, const Model *m, const Ciphertext *ct_dense,
                        const std::vector<const Ciphertext *> &ct_sel)
{
    HCHECK(ct_dense->level == m->lvl_dense, HELRM_E_LEVEL, "ct_dense is not at the model's dense level");
    HCHECK((int)ct_sel.size() == m->n_sel(), HELRM_E_INVAL,
           "the model's selector spans " + std::to_string(m->n_sel()) + " ciphertexts");
    for (auto *s : ct_sel) HCHECK(s->level == m->lvl_sel, HELRM_E_LEVEL, "ct_sel is not at the model's selector level");
    std::unique_ptr<Batch, void (*)(Batch *)> b(batch_create(c, m, {evk}), batch_destroy);
    return model_infer_batch(c, b.get(), {ct_dense}, ct_sel)[0];
}

// client side: pack on the device, encode, encrypt
// ct_dense with `seed`; selector ciphertext k (of n_sel) with seed + 1 + k
void model_encrypt_query(Ctx *c, const EvalKey *evk, const Model *m, const double *dense, const u64 *indices,
                         u64 seed, Ciphertext **ct_dense, std::vector<Ciphertext *> &ct_sel, bool on_device)
{
    const Emb *e = m->emb.get();
    const int ns = m->n_sel();
    const size_t sel_words = ns == 1 ? (size_t)e->in_pad : (size_t)ns * c->n_slots;
    DevMem dd, di, sel(c, sel_words * 8);
    const double *d_dense = dense;
    const u64 *d_idx = indices;
    if (!on_device) {
        for (int t = 0; t < m->T; t++)
            HCHECK(indices[t] < e->cards[t], HELRM_E_INVAL, "index out of range for its table");
        dd = DevMem(c, (size_t)m->n_dense * 8);
        di = DevMem(c, (size_t)m->T * 8);
        CUDA_CHECK(cudaMemcpyAsync(dd.ptr, dense, (size_t)m->n_dense * 8, cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(di.ptr, indices, (size_t)m->T * 8, cudaMemcpyHostToDevice, c->stream));
        d_dense = dd.as<double>();
        d_idx = di.u();
    }
    // the selector ciphertexts on a second stream, the dense one on the context's
    std::vector<std::unique_ptr<Ciphertext>> b;
    Fork branch(c);
    branch.run([&] {
        k::pack_selector(c, sel.as<double>(), d_idx, e->d_tab.as<int>(), m->T, e->base, (int)sel_words);
        for (int k2 = 0; k2 < ns; k2++) {
            // ciphertext k2 holds selector columns [k2 n, k2 n + w) with period pow2ceil(w)
            const int w = ns == 1 ? e->in_pad : std::min(c->n_slots, e->width - k2 * c->n_slots);
            const int per = ns == 1 ? e->in_pad : pow2ceil(w);
            std::unique_ptr<Plaintext> ps(
                pt_encode_dev(c, sel.as<double>() + (size_t)k2 * c->n_slots, w, per, m->lvl_sel, c->delta));
            b.emplace_back(encrypt_pt(c, evk, ps.get(), seed + 1 + k2));
        }
    });
    std::unique_ptr<Plaintext> pd(pt_encode_dev(c, d_dense, m->n_dense, m->p_dense, m->lvl_dense, c->delta));
    std::unique_ptr<Ciphertext> a(encrypt_pt(c, evk, pd.get(), seed));
    branch.join();   // before sel, dd and di (read by the branch) are freed
    *ct_dense = a.release();
    ct_sel.clear();
    for (auto &x : b) ct_sel.push_back(x.release());
}

// model accessors for the C ABI
void model_info(const Model *m, u32 *o)
{
    o[0] = m->lvl_dense;
    o[1] = m->lvl_sel;
    o[2] = m->lvl_z;
    o[3] = m->lvl_u;
    o[4] = m->p_dense;
    o[5] = m->emb->in_pad;
    o[6] = m->W_z;
    o[7] = m->W_u;
    o[8] = (u32)const_cast<Model *>(m)->plaintexts().size();
    o[9] = (u32)m->n_sel();
}
std::vector<int> model_rotations(const Model *m) { return m->rotations(); }

// The highest level at which the model uses each rotation (baby and giant
// steps at the matvec's level, folds one level lower, after its rescale; the
// interaction's rotations at lvl_z - 1, after the mask rescale) and the
// highest level of a relinearisation (the first x^2 of the bottom MLP).
std::vector<std::pair<int, int>> model_key_levels(const Model *m, int *relin_level)
{
    std::map<int, int> lv;
    auto use = [&](int st, int l) {
        auto it = lv.find(st);
        if (it == lv.end() || it->second < l) lv[st] = l;
    };
    auto mat = [&](const PtMatrix *pm) {
        if (!pm) return;
        for (auto &gb : pm->gb) {
            if (gb.second) use(gb.second, pm->level);
            if (gb.first) use(gb.first * pm->n1, pm->level);
        }
        for (auto &f : pm->folds)
            for (int dd = 1; dd < f.second; dd++) use(dd * f.first, pm->level - 1);
    };
    int rl = -1;
    for (auto &L : m->bottom) {
        mat(L.pm.get());
        if (L.square) rl = std::max(rl, L.pm->level - 1);
    }
    mat(m->emb->pm.get());
    for (auto &ch : m->emb->chunks) mat(ch.get());
    if (m->interaction == 0) {
        use(-DIM * m->Bp, m->lvl_z - 1);
        for (int s = 1; s <= m->S; s++) use(DIM * s, m->lvl_z - 1);
        rl = std::max(rl, m->lvl_z - 1);
    }
    for (auto &L : m->top) {
        mat(L.pm.get());
        if (L.square) rl = std::max(rl, L.pm->level - 1);
    }
    // a bootstrap works at the top of the chain (its keys at full level)
    for (const Model::BootPoint *bp : m->boot_points()) {
        for (int st : bp->b->rotations()) use(st, m->ctx->L);
        rl = m->ctx->L;
    }
    *relin_level = std::max(rl, 0);
    return std::vector<std::pair<int, int>>(lv.begin(), lv.end());
}
const PtMatrix *emb_matrix_of(const Emb *e) { return e->pm.get(); }
int emb_n_chunks(const Emb *e) { return e->pm ? 1 : (int)e->chunks.size(); }
PtMatrix *emb_chunk(const Emb *e, int c) { return e->pm ? e->pm.get() : e->chunks[c].get(); }
int emb_chunk_period(const Emb *e, int c) { return e->pm ? e->in_pad : e->chunks[c]->in_pad; }

// y = M s = sum_c M_c s_c for a selector spread over several ciphertexts
Ciphertext *emb_lookup_multi(Ctx *c, const EvalKey *evk, const Emb *e, const std::vector<const Ciphertext *> &sel)
{
    const int n = emb_n_chunks(e);
    HCHECK((int)sel.size() == n, HELRM_E_INVAL,
           "the selector spans " + std::to_string(n) + " ciphertexts, got " + std::to_string(sel.size()));
    // chunks of one shape share their giant steps (matvec_sum); the groups, in
    // order of first appearance, are added in order
    std::vector<std::vector<int>> groups;
    for (int k = 0; k < n; k++) {
        bool placed = false;
        for (auto &grp : groups)
            if (same_shape(emb_chunk(e, grp[0]), emb_chunk(e, k))) {
                grp.push_back(k);
                placed = true;
                break;
            }
        if (!placed) groups.push_back({k});
    }
    std::unique_ptr<Ciphertext> y;
    for (auto &grp : groups) {
        std::vector<const PtMatrix *> ms;
        std::vector<const Ciphertext *> xs;
        for (int k : grp) {
            ms.push_back(emb_chunk(e, k));
            xs.push_back(sel[k]);
        }
        std::unique_ptr<Ciphertext> t(matvec_sum(c, evk, ms, xs));
        y.reset(y ? ct_add(c, y.get(), t.get()) : t.release());
    }
    return y.release();
}
void emb_info(const Emb *e, u32 *width, u32 *period)
{
    *width = e->width;
    *period = e->in_pad;
}
Ctx *emb_ctx(const Emb *e) { return e->ctx; }
Ctx *model_ctx(const Model *m) { return m->ctx; }
u32 model_n_dense(const Model *m) { return (u32)m->n_dense; }
u32 model_n_tables(const Model *m) { return (u32)m->T; }
int model_n_sel(const Model *m) { return m->n_sel(); }

}  // namespace helrm
