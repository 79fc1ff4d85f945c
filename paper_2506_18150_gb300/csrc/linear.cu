// linear.cu -- plaintext-matrix x ciphertext-vector products (HE-LRM Sec. 2.1.4
// and Sec. 3.2.1: diagonal method with baby-step giant-step, double hoisting).
//
// Layout: a vector of padded length v is replicated with period v over the n
// slots.  For W padded to out_pad x in_pad there are D = min(in_pad, out_pad)
// extended diagonals diag_i[j] = W[j mod out_pad, (j + i) mod in_pad]; when the
// matrix is wide, rotate-and-add folds by in_pad/2, ..., out_pad finish the
// sum (levels of up to 3 hoisted rotations: rot(y, d stride) for d < 4,
// stride out_pad, 4 out_pad, 16 out_pad, ...).  BSGS: n1 = min(D, max(16, D / 8)), n2 = D / n1 <= 8 (a hoisted baby
// step costs a key inner product and a key read, a giant step a ModDown and a
// ModUp as well), i = g n1 + b, diag'_{g,b} = rot(diag_i, -g n1), which reads
// W[(j - g n1) mod out_pad, (j + b) mod in_pad].
//
// Double hoisting: one ModUp of c1; each baby step b is phi_{5^b} applied to
// the extended digits, the key inner product and P phi(c0), all kept over QP
// (no ModDown); one MAC kernel forms inner_g = sum_b diag'_{g,b} baby_b for all
// g; each giant step g > 0 ModDowns the a-part of inner_g, ModUps it, applies
// phi_{5^{g n1}} and the key, and adds phi(b-part); one ModDown at the end,
// then rescale, then the folds.
#include <algorithm>
#include <cmath>

#include "core.cuh"

namespace helrm {

int pow2ceil(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

std::vector<int> PtMatrix::rotations() const
{
    std::vector<int> st;
    for (auto &gb2 : gb) {
        if (gb2.second) st.push_back(gb2.second);
        if (gb2.first) st.push_back(gb2.first * n1);
    }
    for (auto &f : folds)
        for (int d = 1; d < f.second; d++) st.push_back(d * f.first);
    std::sort(st.begin(), st.end());
    st.erase(std::unique(st.begin(), st.end()), st.end());
    return st;
}

void PtMatrix::upload_index()
{
    std::vector<const u64 *> ptrs;
    for (auto &p : pts) ptrs.push_back(p->data.u());
    std::vector<int> idx((size_t)n1 * n2, -1);
    for (size_t t = 0; t < gb.size(); t++) idx[(size_t)gb[t].first * n1 + gb[t].second] = (int)t;
    d_ptrs = DevMem(ctx, std::max<size_t>(ptrs.size(), 1) * sizeof(u64 *));
    d_gb_index = DevMem(ctx, idx.size() * sizeof(int));
    if (!ptrs.empty())
        CUDA_CHECK(cudaMemcpyAsync(d_ptrs.ptr, ptrs.data(), ptrs.size() * sizeof(u64 *), cudaMemcpyHostToDevice,
                                   ctx->stream));
    CUDA_CHECK(cudaMemcpyAsync(d_gb_index.ptr, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice,
                               ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
}

PtMatrix *ptmat_prepare(Ctx *c, const double *W, int rows, int cols, int in_pad, int out_pad, int level,
                        double ct_scale, double target_scale)
{
    HCHECK(level >= 1 && level <= c->L, HELRM_E_LEVEL, "matvec level must be in [1, L]");
    return ptmat_prepare_scaled(c, W, nullptr, rows, cols, in_pad, out_pad, level,
                                (double)c->primes[level] * target_scale / ct_scale, target_scale);
}

PtMatrix *ptmat_prepare_scaled(Ctx *c, const double *W, const double *W_im, int rows, int cols, int in_pad,
                               int out_pad, int level, double pt_scale, double out_scale)
{
    HCHECK(W && rows >= 1 && cols >= 1, HELRM_E_INVAL, "empty matrix");
    HCHECK(in_pad == pow2ceil(in_pad) && out_pad == pow2ceil(out_pad), HELRM_E_INVAL, "pads must be powers of two");
    HCHECK(rows <= out_pad && cols <= in_pad, HELRM_E_INVAL, "matrix larger than its padding");
    HCHECK(in_pad <= c->n_slots && out_pad <= c->n_slots, HELRM_E_PARAM, "padding exceeds the slot count");
    HCHECK(level >= 1 && level <= c->L, HELRM_E_LEVEL, "matvec level must be in [1, L]");
    std::unique_ptr<PtMatrix> m(new PtMatrix(c));
    m->in_pad = in_pad;
    m->out_pad = out_pad;
    m->D = std::min(in_pad, out_pad);
    m->n1 = std::min(m->D, std::max(16, m->D / 8));   // at most 8 giant steps
    m->n2 = m->D / m->n1;
    m->level = level;
    // folds: levels of up to 3 hoisted rotations (radix 4), from the smallest stride,
    // together summing rot(y, j out_pad) over j < in_pad / out_pad
    const int fold = in_pad > out_pad ? in_pad / out_pad : 1;   // a tall matrix has no folds
    for (int bits = 31 - __builtin_clz((unsigned)fold), stride = out_pad; bits > 0;) {
        const int r = std::min(2, bits);
        m->folds.push_back({stride, 1 << r});
        stride <<= r;
        bits -= r;
    }
    m->pt_scale = pt_scale;
    m->out_scale = out_scale;
    auto Wp = [&](const double *A, int r, int col) -> double {
        return (r < rows && col < cols) ? A[(size_t)r * cols + col] : 0.0;
    };
    const int P = std::max(in_pad, out_pad);
    std::vector<double> v(P), vi(W_im ? P : 0);
    for (int g = 0; g < m->n2; g++)
        for (int b = 0; b < m->n1; b++) {
            bool nz = false;
            for (int j = 0; j < P; j++) {
                int r = ((j - g * m->n1) % out_pad + out_pad) % out_pad;
                v[j] = Wp(W, r, (j + b) % in_pad);
                nz |= v[j] != 0.0;
                if (W_im) {
                    vi[j] = Wp(W_im, r, (j + b) % in_pad);
                    nz |= vi[j] != 0.0;
                }
            }
            if (!nz) continue;
            m->gb.push_back({g, b});
            m->pts.emplace_back(pt_encode(c, v.data(), P, P, level, true, m->pt_scale, PT_MONT,
                                          W_im ? vi.data() : nullptr));
        }
    c->check_device_errors();
    m->upload_index();
    return m.release();
}

// The baby-step half of a product (one ModUp of c1, the hoisted baby steps
// and the BSGS MAC over QP): inner[g][2][plane] for every giant step g with
// diagonals (need_g[g] set).
static void baby_products(Ctx *c, const EvalKey *evk, const PtMatrix *m, const Ciphertext *in, u64 *inner,
                          std::vector<char> &need_g)
{
    const int l = in->level, N = c->N, nq = l + 1, nl = nq + c->K, dnum = c->dnum(l);
    HCHECK(l == m->level, HELRM_E_LEVEL, "ciphertext level does not match the prepared matrix");
    const size_t plane = (size_t)nl * N;
    std::vector<char> need_b(m->n1, 0);
    need_g.assign(m->n2, 0);
    for (auto &gb : m->gb) {
        need_b[gb.second] = 1;
        need_g[gb.first] = 1;
    }
    // keys first, so a missing key fails before any work
    std::vector<const SwitchKey *> bkey(m->n1, nullptr);
    for (int b = 1; b < m->n1; b++)
        if (need_b[b]) bkey[b] = rot_key(evk, c->galois(b), l);
    for (int g = 1; g < m->n2; g++)
        if (need_g[g]) rot_key(evk, c->galois(g * m->n1), l);

    DevMem digits(c, (size_t)dnum * plane * 8);
    bool any_baby = false;
    for (int b = 1; b < m->n1; b++) any_baby |= need_b[b] != 0;
    if (any_baby) ks_modup(c, in->c1(), l, digits.u());   // hoisted: one ModUp for all baby steps
    if (m->n1 <= 64 && m->n2 <= 8) {
        // baby steps formed in registers inside the MAC (no baby buffer)
        std::vector<u64> gals(m->n1, 1);
        for (int b = 1; b < m->n1; b++)
            if (need_b[b]) gals[b] = c->galois(b);
        k::bsgs_tma(c, inner, digits.u(), in->c0(), in->c1(), bkey.data(), gals.data(),
                    m->d_ptrs.as<const u64 *>(), m->d_gb_index.as<int>(), (int)m->gb.size(), m->n1, m->n2, l);
    } else {
        // wide baby-step sets: baby steps materialised over QP, then the tiled MAC
        DevMem baby(c, (size_t)m->n1 * 2 * plane * 8);
        for (int b = 0; b < m->n1; b++) {
            if (!need_b[b]) continue;
            u64 *bb = baby.u() + (size_t)b * 2 * plane;
            if (b == 0) {   // (P c0, P c1) over QP: P mod q_i on the Q limbs, 0 on the P limbs
                for (int p = 0; p < 2; p++) {
                    k::mul_scalar_mont(c, bb + p * plane, p ? in->c1() : in->c0(), c->d_pmod_mont.u(), nq,
                                       c->qmap(l));
                    k::zero(c, bb + p * plane + (size_t)nq * N, (size_t)c->K * N);
                }
            } else {
                k::ks_inner_auto(c, bb, digits.u(), dnum, bkey[b], l, c->galois(b), in->c0(),
                                 c->d_pmod_mont.u());
            }
        }
        k::bsgs_mac(c, inner, baby.u(), (int)m->gb.size(), m->d_ptrs.as<const u64 *>(), m->d_gb_index.as<int>(),
                    m->n2, m->n1, nl, c->qmap(l));
    }
}

// The giant-step half: the giant steps on the QP inner products, one ModDown
// of their sum, the rescale (scale: the product's scale before it) and the
// folds of a wide matrix.
static Ciphertext *giant_steps(Ctx *c, const EvalKey *evk, const PtMatrix *m, u64 *inner,
                               const std::vector<char> &need_g, int l, double scale)
{
    const int N = c->N, nq = l + 1, nl = nq + c->K, dnum = c->dnum(l);
    const size_t plane = (size_t)nl * N;
    std::vector<const SwitchKey *> gkey(m->n2, nullptr);
    for (int g = 1; g < m->n2; g++)
        if (need_g[g]) gkey[g] = rot_key(evk, c->galois(g * m->n1), l);
    DevMem digits(c, (size_t)dnum * plane * 8);
    // the giant steps accumulate into inner_0
    u64 *acc = inner;
    DevMem c1q(c, (size_t)nq * N * 8);
    if (!need_g[0]) k::zero(c, acc, 2 * plane);
    for (int g = 1; g < m->n2; g++) {
        if (!need_g[g]) continue;
        const u64 *ig = inner + (size_t)g * 2 * plane;
        // giant step on a QP ciphertext: ModDown the a-part, ModUp, then one kernel
        // adds the key inner product and phi of the b-part (already over QP) to acc
        const u64 gal = c->galois(g * m->n1);
        ks_moddown(c, ig + plane, l, c1q.u());
        ks_modup(c, c1q.u(), l, digits.u());
        k::ks_inner_auto(c, acc, digits.u(), dnum, gkey[g], l, gal, nullptr, nullptr, ig, true);
    }
    std::unique_ptr<Ciphertext> o(new_ct(c, l, scale));
    ks_moddown2(c, acc, l, o->c0(), o->c1());
    std::unique_ptr<Ciphertext> y(ct_rescale(c, o.get()));
    y->scale = m->out_scale;
    for (auto &f : m->folds) {
        std::vector<int> steps;
        for (int d = 1; d < f.second; d++) steps.push_back(d * f.first);
        std::vector<Ciphertext *> rs;
        ct_rotate_hoisted(c, evk, y.get(), steps, rs);
        std::vector<std::unique_ptr<Ciphertext>> own;
        for (auto *r : rs) own.emplace_back(r);
        std::unique_ptr<Ciphertext> acc2(ct_add(c, y.get(), own[0].get()));
        for (size_t i = 1; i < own.size(); i++) acc2.reset(ct_add(c, acc2.get(), own[i].get()));
        y = std::move(acc2);
    }
    return y.release();
}

Ciphertext *matvec(Ctx *c, const EvalKey *evk, const PtMatrix *m, const Ciphertext *in)
{
    const int l = in->level;
    const size_t plane = (size_t)(l + 1 + c->K) * c->N;
    DevMem inner(c, (size_t)m->n2 * 2 * plane * 8);
    std::vector<char> need_g;
    baby_products(c, evk, m, in, inner.u(), need_g);
    return giant_steps(c, evk, m, inner.u(), need_g, l, in->scale * m->pt_scale);
}

bool same_shape(const PtMatrix *a, const PtMatrix *b)
{
    return a->in_pad == b->in_pad && a->out_pad == b->out_pad && a->D == b->D && a->n1 == b->n1 &&
           a->n2 == b->n2 && a->level == b->level && a->folds == b->folds && a->pt_scale == b->pt_scale &&
           a->out_scale == b->out_scale;
}

// sum_k W_k x_k for matrices of one shape (reading R31): the baby-step
// products are added over QP, giant step by giant step, and the sum takes one
// set of giant steps, one ModDown, one rescale and one set of folds.
Ciphertext *matvec_sum(Ctx *c, const EvalKey *evk, const std::vector<const PtMatrix *> &ms,
                       const std::vector<const Ciphertext *> &in)
{
    HCHECK(!ms.empty() && ms.size() == in.size(), HELRM_E_INVAL, "matvec_sum takes one ciphertext per matrix");
    if (ms.size() == 1) return matvec(c, evk, ms[0], in[0]);
    const int l = in[0]->level;
    for (size_t k2 = 0; k2 < ms.size(); k2++) {
        HCHECK(same_shape(ms[k2], ms[0]), HELRM_E_PARAM, "matvec_sum: the matrices differ in shape");
        HCHECK(in[k2]->level == l && in[k2]->scale == in[0]->scale, HELRM_E_SCALE,
               "matvec_sum: the ciphertexts differ in level or scale");
    }
    const PtMatrix *m = ms[0];
    const int nl = l + 1 + c->K;
    const size_t plane = (size_t)nl * c->N, words = (size_t)m->n2 * 2 * plane;
    DevMem total(c, words * 8), part(c, words * 8);
    k::zero(c, total.u(), words);
    std::vector<char> need_all(m->n2, 0), need_g;
    for (size_t k2 = 0; k2 < ms.size(); k2++) {
        k::zero(c, part.u(), words);
        baby_products(c, evk, ms[k2], in[k2], part.u(), need_g);
        for (int g = 0; g < m->n2; g++) need_all[g] |= need_g[g];
        k::add(c, total.u(), total.u(), part.u(), m->n2 * 2 * nl, c->qmap(l, 0, nl));
    }
    return giant_steps(c, evk, m, total.u(), need_all, l, in[0]->scale * m->pt_scale);
}

}  // namespace helrm
