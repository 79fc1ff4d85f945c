// boot.cu -- bootstrapping: a ciphertext at the bottom of the chain gets its
// levels back (HE-LRM Sec. 2.1.4; the paper's Criteo models with polynomial
// ReLU / SiLU activations need 12 or 5 of them, Sec. 5.4).  The paper names
// the parts (ModRaise, CoeffToSlot, EvalMod, SlotToCoeff) but not their
// steps; this is the standard pipeline for a ciphertext whose real slot
// vector is periodic with period n_s (2 n_s <= n), under a secret with h
// non-zero coefficients:
//
//   1. boost: at level 0 the ciphertext is multiplied by the integer 2^b, so
//      the message m = 2^b scale z stays a small fraction of q_0;
//   2. ModRaise: c0, c1 mod q_0, centred, become residues of every prime of
//      the top level L (decrypting to m + q_0 I over Q_L, |I_k| <= (h+1)/2);
//   3. SubSum: ct += rot(ct, n_s 2^i), i < log2(n / n_s): the trace onto
//      Z[Y], Y = X^g, g = N / (2 n_s);
//   4. CoeffToSlot: with U[i][k] = xi^(k 5^i), xi = exp(i pi / (2 n_s)), the
//      2 n_s coefficients t of the polynomial in Y are (U^H w + U^T conj(w)) /
//      (2 n_s) for its n_s slot values w; the second term is the conjugate
//      of the first, so one BSGS product C = U^H w / (2 n_s) and its
//      conjugate (X -> X^(2N-1)) give t = C + conj(C), and the slots
//      (period 2 n_s) hold u_k / 2^r, u_k = m_k / q_0 + I_k, at about
//      eval_scale after cts_levels rescales;
//   5. EvalMod: y - 1 / (4 2^r) (a constant), a polynomial fit of
//      cos(2 pi y) on |y| <= (K + 1/2) / 2^r, then r double angles
//      c <- 2 c^2 - 1: c = cos(2 pi (u - 1/4)) = sin(2 pi u), about
//      2 pi m_k / q_0;
//   6. SlotToCoeff: z = U (q_0 / (2 pi 2^b s_ref)) c, a BSGS product from
//      period 2 n_s to period n_s (one fold).
//
// Every step is an exact integer operation of the scheme; only the constants
// (diagonals, the polynomial, the scales) come from FP64.  On the
// bootstrappable chain (the top primes 60-bit) EvalMod runs at a scale of
// about 2^60, so the noise the double angles multiply stays far below the
// message; the output sits cts_levels + depth + r + 1 levels below L.
#include <cmath>

#include "model.cuh"

namespace helrm {

namespace {

// U[i][k] = exp(i pi ((5^i mod 4 n_s) k mod 4 n_s) / (2 n_s)), i < n_s, k < 2 n_s
void slot_matrix(int n_s, std::vector<double> &re, std::vector<double> &im)
{
    const long long M = 4LL * n_s;
    re.assign((size_t)n_s * 2 * n_s, 0.0);
    im.assign(re.size(), 0.0);
    long long e = 1;
    for (int i = 0; i < n_s; i++) {
        for (int k = 0; k < 2 * n_s; k++) {
            const long long t = (e * k) % M;
            const double ang = M_PI * (double)t / (2.0 * n_s);
            re[(size_t)i * 2 * n_s + k] = std::cos(ang);
            im[(size_t)i * 2 * n_s + k] = std::sin(ang);
        }
        e = e * 5 % M;
    }
}

}  // namespace

// Interpolant of cos(2 pi y) at the degree + 1 Chebyshev points (first kind)
// of [-Y, Y], Y = (K + 1/2) / 2^r, in the power basis of y; odd coefficients
// (zero for an even function) set to exact zeros.
std::vector<double> boot_cos_fit(int K, int r, int degree)
{
    HCHECK(degree >= 2 && degree % 2 == 0 && degree <= 64, HELRM_E_INVAL, "the cosine fit needs an even degree");
    const int n = degree + 1;
    const double Y = (K + 0.5) / std::ldexp(1.0, r);
    std::vector<double> f(n), t(n);
    for (int j = 0; j < n; j++) {
        t[j] = std::cos(M_PI * (j + 0.5) / n);
        f[j] = std::cos(2.0 * M_PI * Y * t[j]);
    }
    // Chebyshev coefficients c_k = (2/n) sum_j f_j T_k(t_j), c_0 halved
    std::vector<double> ch(n, 0.0);
    for (int k = 0; k < n; k++) {
        double s = 0;
        for (int j = 0; j < n; j++) s += f[j] * std::cos(k * M_PI * (j + 0.5) / n);
        ch[k] = (k == 0 ? 1.0 : 2.0) * s / n;
    }
    // power basis in t: T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1}
    std::vector<double> a(n, 0.0), tp(n, 0.0), tc(n, 0.0), tn(n, 0.0);
    tp[0] = 1.0;
    a[0] += ch[0];
    if (n > 1) {
        tc[1] = 1.0;
        a[1] += ch[1];
    }
    for (int k = 2; k < n; k++) {
        for (int i = 0; i < n; i++) tn[i] = (i ? 2.0 * tc[i - 1] : 0.0) - tp[i];
        for (int i = 0; i < n; i++) a[i] += ch[k] * tn[i];
        tp.swap(tc);
        tc.swap(tn);
    }
    // t = y / Y
    double sc = 1.0;
    for (int i = 0; i < n; i++) {
        a[i] = (i % 2) ? 0.0 : a[i] / sc;
        sc *= Y;
    }
    return a;
}

std::vector<int> Boot::rotations() const
{
    std::vector<int> st = subsum_steps;
    for (PtMatrix *m : matrices()) {
        auto r = m->rotations();
        st.insert(st.end(), r.begin(), r.end());
    }
    std::sort(st.begin(), st.end());
    st.erase(std::unique(st.begin(), st.end()), st.end());
    return st;
}

Boot *boot_create(Ctx *c, const BootDesc &d)
{
    const int n_s = d.n_s, L = c->L;
    HCHECK(n_s >= 1 && (n_s & (n_s - 1)) == 0 && 2 * n_s <= c->n_slots, HELRM_E_INVAL,
           "n_s must be a power of two with 2 n_s <= N/2");
    HCHECK(d.r >= 0 && d.r <= 20 && d.K >= 1 && d.log2_boost >= 0 && d.log2_boost <= 30, HELRM_E_INVAL,
           "bootstrapping parameters out of range");
    HCHECK(d.cts_levels == 1 || d.cts_levels == 2, HELRM_E_INVAL, "CoeffToSlot takes one or two rescales");
    HCHECK(d.s_ref > 0 && d.eval_scale > 0, HELRM_E_INVAL, "scales must be positive");
    std::unique_ptr<Boot> b(new Boot(c));
    b->n_s = n_s;
    b->K = d.K;
    b->r = d.r;
    b->degree = d.degree;
    b->log2_boost = d.log2_boost;
    b->cts_levels = d.cts_levels;
    b->s_ref = d.s_ref;
    b->eval_scale = d.eval_scale;
    b->coeffs = d.coeffs.empty() ? boot_cos_fit(d.K, d.r, d.degree) : d.coeffs;
    HCHECK((int)b->coeffs.size() == d.degree + 1 && b->coeffs.back() != 0.0, HELRM_E_INVAL,
           "the cosine polynomial must have degree + 1 coefficients and a non-zero leading one");
    const int used = d.cts_levels + poly_depth(d.degree) + d.r + 1;
    HCHECK(used <= L, HELRM_E_PARAM, "the chain is too short for this bootstrapping");
    b->level_top = L;
    b->level_stc = L - used + 1;
    b->level_out = L - used;
    const int g = c->N / (2 * n_s);
    std::vector<double> ure, uim;
    slot_matrix(n_s, ure, uim);
    // CoeffToSlot: A = f U^H (2 n_s x n_s), f = 1 / (2 n_s g 2^r)
    const double f = 1.0 / (2.0 * n_s * g * std::ldexp(1.0, d.r));
    double pt_cts = d.eval_scale;
    for (int i = 0; i < d.cts_levels; i++) pt_cts *= (double)c->primes[L - i];
    pt_cts /= (double)c->primes[0];
    const double out_cts = (double)c->primes[0] * pt_cts / (double)c->primes[L];
    std::vector<double> are((size_t)2 * n_s * n_s), aim(are.size());
    for (int k = 0; k < 2 * n_s; k++)
        for (int i = 0; i < n_s; i++) {
            are[(size_t)k * n_s + i] = f * ure[(size_t)i * 2 * n_s + k];
            aim[(size_t)k * n_s + i] = f * -uim[(size_t)i * 2 * n_s + k];
        }
    b->cts_a.reset(ptmat_prepare_scaled(c, are.data(), aim.data(), 2 * n_s, n_s, n_s, 2 * n_s, L, pt_cts, out_cts));
    // SlotToCoeff: S = (q_0 / (2 pi 2^b s_ref)) U (n_s x 2 n_s), from about eval_scale to Delta
    const int ls = b->level_stc;
    const double fs = (double)c->primes[0] / (2.0 * M_PI * std::ldexp(1.0, d.log2_boost) * d.s_ref);
    std::vector<double> sre(ure.size()), sim(ure.size());
    for (size_t t = 0; t < ure.size(); t++) {
        sre[t] = fs * ure[t];
        sim[t] = fs * uim[t];
    }
    b->stc.reset(ptmat_prepare_scaled(c, sre.data(), sim.data(), n_s, 2 * n_s, 2 * n_s, n_s, ls,
                                      (double)c->primes[ls] * c->delta / d.eval_scale, c->delta));
    for (int s = n_s; s < c->n_slots; s <<= 1) b->subsum_steps.push_back(s);
    b->boost_mont = int_table(c, (i64)1 << d.log2_boost, true);
    // the scales every later step will see (the same FP64 operations as the run)
    double sc = out_cts;
    int lv = L - 1;
    for (int i = 1; i < d.cts_levels; i++) sc = sc / (double)c->primes[lv--];
    b->s_cts = sc;
    b->c_shift = int_table_f(c, round_half_away(-sc / (4.0 * std::ldexp(1.0, d.r))), false);
    b->plan.reset(act_plan(c, b->coeffs, lv, sc, d.eval_scale));
    sc = b->plan->out_scale;
    lv = b->plan->out_level;
    for (int i = 0; i < d.r; i++) {
        sc = (sc * sc) / (double)c->primes[lv--];
        b->c_double.push_back(int_table_f(c, round_half_away(-sc), false));
    }
    HCHECK(lv == ls, HELRM_E_PARAM, "internal: the EvalMod levels do not meet SlotToCoeff");
    b->s_eval = sc;
    b->c_out = (sc * b->stc->pt_scale) / (double)c->primes[ls];
    return b.release();
}

namespace {

// a + v on every slot (the integer v in coefficient 0: v on every NTT value of
// c0), v given as its residues per prime id
Ciphertext *ct_add_int(Ctx *c, const Ciphertext *a, const DevMem &t)
{
    std::unique_ptr<Ciphertext> o(new_ct(c, a->level, a->scale));
    k::add_scalar(c, o->c0(), a->c0(), t.u(), a->level + 1, c->qmap(a->level));
    k::copy(c, o->c1(), a->c1(), (size_t)(a->level + 1) * c->N);
    return o.release();
}

}  // namespace

Ciphertext *bootstrap(Ctx *c, const EvalKey *evk, const Boot *b, const Ciphertext *in,
                      std::vector<Ciphertext *> *stages)
{
    using P = std::unique_ptr<Ciphertext>;
    const int N = c->N, L = b->level_top;
    const double in_scale = in->scale;
    auto stage = [&](P &x) {
        if (stages) stages->push_back(ct_drop(c, x.get(), x->level));
    };
    // 1. level 0, times 2^b
    P x0(ct_drop(c, in, 0));
    k::mul_scalar_mont(c, x0->data.u(), x0->data.u(), b->boost_mont.u(), 2, c->qmap(0, 0, 1));
    x0->scale = in_scale * std::ldexp(1.0, b->log2_boost);
    // 2. ModRaise: both limbs to coefficients, centred mod q_0, residues of q_0..q_L, back to NTT
    DevMem coef(c, (size_t)2 * N * 8);
    std::vector<k::NttLimb> inv = {{x0->c0(), coef.u(), 0, nullptr, nullptr},
                                   {x0->c1(), coef.u() + N, 0, nullptr, nullptr}};
    k::ntt_run(c, inv, true, nullptr);
    P x(new_ct(c, L, (double)c->primes[0]));
    k::mod_raise(c, x->data.u(), coef.u(), (size_t)N, 2, L + 1, c->qmap(L));
    k::ntt_fwd(c, x->data.u(), 2 * (L + 1), c->qmap(L, 0, L + 1));
    stage(x);
    // 3. SubSum
    for (int st : b->subsum_steps) {
        P r(ct_rotate(c, evk, x.get(), st));
        x.reset(ct_add(c, x.get(), r.get()));
    }
    stage(x);
    // 4. CoeffToSlot: C = A w, then C + conj(C)
    P y(matvec(c, evk, b->cts_a.get(), x.get()));
    {
        P yc(ct_apply_galois(c, evk, y.get(), 2ull * N - 1));
        y.reset(ct_add(c, y.get(), yc.get()));
    }
    for (int i = 1; i < b->cts_levels; i++) y.reset(ct_rescale(c, y.get()));
    stage(y);
    // 5. EvalMod
    HCHECK(y->scale == b->s_cts && y->level == b->plan->in_level, HELRM_E_SCALE,
           "internal: CoeffToSlot ended on another scale or level");
    y.reset(ct_add_int(c, y.get(), b->c_shift));
    P cv(poly_b(c, {evk}, {y.get()}, *b->plan)[0]);
    for (int i = 0; i < b->r; i++) {
        cv.reset(ct_mul(c, evk, cv.get(), cv.get()));
        cv.reset(ct_add(c, cv.get(), cv.get()));
        cv.reset(ct_add_int(c, cv.get(), b->c_double[i]));
    }
    stage(cv);
    // 6. SlotToCoeff; the declared scale makes the slots decode to the input's values
    HCHECK(cv->level == b->level_stc && cv->scale == b->s_eval, HELRM_E_LEVEL,
           "internal: EvalMod ended on another level or scale");
    P z(matvec(c, evk, b->stc.get(), cv.get()));
    z->scale = b->out_scale(in_scale);
    if (stages) stages->push_back(ct_drop(c, z.get(), z->level));
    return z.release();
}

}  // namespace helrm
