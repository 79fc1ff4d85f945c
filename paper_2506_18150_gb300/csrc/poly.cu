// poly.cu -- homomorphic evaluation of a real polynomial on ciphertexts: the
// activations of the paper's Criteo models are polynomial approximations of
// ReLU and SiLU (HE-LRM Sec. 2.1.4, Sec. 5.4).
//
// The paper fixes neither the coefficients nor the evaluation schedule; the
// schedule is:
//   - powers: x^k = x^a * x^(k-a), a the largest power of two below k (a
//     ct x ct product: tensor, relinearise, rescale, operands first taken to
//     the lower of their levels), so x^k sits ceil(log2 k) levels below x;
//     only the powers that a non-zero a_k needs (with their operands) are
//     formed, in increasing k;
//   - terms: each x^k with a_k != 0 is taken to the level L_c of the deepest
//     power and multiplied by the integer c_k = round_half_away(a_k s_k),
//     s_k = (target q_{L_c}) / scale(x^k) (so every term carries the scale
//     target q_{L_c}); the terms are added in increasing k;
//   - one rescale, then a_0 as the integer round_half_away(a_0 scale) in every
//     slot (a constant polynomial).
// A degree-d polynomial consumes ceil(log2 d) + 1 levels.  Everything but
// the FP64 products that fix s_k and c_k is exact integer arithmetic.
#include <cmath>

#include "model.cuh"

namespace helrm {
namespace {

u64 mod_signed(i64 v, u64 q)
{
    const u64 m = (u64)(v < 0 ? -(v + 1) : v) % q;   // |v| without overflow at INT64_MIN
    if (v >= 0) return m;
    const u64 r = (m + 1) % q;                       // |v| mod q
    return r ? q - r : 0;
}

u64 mulmod_host(u64 a, u64 b, u64 q) { return (u64)(((unsigned __int128)a * b) % q); }

}  // namespace

// per-prime residues of an integer (plain, or times R for Montgomery products)
DevMem int_table(Ctx *c, i64 v, bool mont)
{
    std::vector<u64> t(c->nP());
    for (int i = 0; i < c->nP(); i++) {
        const u64 r = mod_signed(v, c->primes[i]);
        t[i] = mont ? mulmod_host(r, c->pinfo[i].rmod, c->primes[i]) : r;
    }
    DevMem d(c, t.size() * 8);
    CUDA_CHECK(cudaMemcpyAsync(d.ptr, t.data(), t.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    return d;
}

double round_half_away(double v) { return std::copysign(std::floor(std::fabs(v) + 0.5), v); }

// the same for an integer-valued double of any finite size: v = m 2^e with an
// integer mantissa m (|m| < 2^53), so v mod q = m (2^e mod q) mod q, exactly
DevMem int_table_f(Ctx *c, double v, bool mont)
{
    HCHECK(std::isfinite(v) && v == std::floor(v), HELRM_E_INVAL, "internal: constant is not an integer");
    if (std::fabs(v) < 9.2e18) return int_table(c, (i64)v, mont);
    int e = 0;
    const double f = std::frexp(std::fabs(v), &e);   // |v| = f 2^e, f in [0.5, 1)
    const u64 m = (u64)std::ldexp(f, 53);
    e -= 53;                                         // |v| = m 2^e, e > 0 here
    std::vector<u64> t(c->nP());
    for (int i = 0; i < c->nP(); i++) {
        const u64 q = c->primes[i];
        u64 p2 = 1, b = 2 % q;
        for (int k = e; k; k >>= 1, b = mulmod_host(b, b, q))
            if (k & 1) p2 = mulmod_host(p2, b, q);
        u64 r = mulmod_host(m % q, p2, q);
        if (v < 0 && r) r = q - r;
        t[i] = mont ? mulmod_host(r, c->pinfo[i].rmod, q) : r;
    }
    DevMem d(c, t.size() * 8);
    CUDA_CHECK(cudaMemcpyAsync(d.ptr, t.data(), t.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    return d;
}

int poly_power_depth(int k) { return k <= 1 ? 0 : 32 - __builtin_clz((unsigned)(k - 1)); }
int poly_depth(int d) { return d <= 0 ? 0 : poly_power_depth(d) + 1; }

ActPlan *act_plan(Ctx *c, const std::vector<double> &a, int level, double scale, double target)
{
    const int d = (int)a.size() - 1;
    HCHECK(d >= 1 && a[d] != 0.0, HELRM_E_INVAL, "need a non-constant polynomial with a non-zero leading coefficient");
    for (double v : a) HCHECK(std::isfinite(v), HELRM_E_INVAL, "polynomial coefficients must be finite");
    HCHECK(level >= poly_depth(d) && level <= c->L, HELRM_E_LEVEL,
           "a degree-" + std::to_string(d) + " polynomial needs " + std::to_string(poly_depth(d)) + " levels");
    std::unique_ptr<ActPlan> p(new ActPlan());
    p->a = a;
    p->in_level = level;
    p->in_scale = scale;
    // the powers a non-zero coefficient needs, with their operands
    std::vector<char> need(d + 1, 0);
    std::vector<int> stack;
    for (int k = 2; k <= d; k++)
        if (a[k] != 0.0) stack.push_back(k);
    while (!stack.empty()) {
        const int k = stack.back();
        stack.pop_back();
        if (k < 2 || need[k]) continue;
        need[k] = 1;
        const int x = 1 << (poly_power_depth(k) - 1);
        stack.push_back(x);
        stack.push_back(k - x);
    }
    std::map<int, int> lv{{1, level}};
    p->pw_scale[1] = scale;
    for (int k = 2; k <= d; k++) {
        if (!need[k]) continue;
        const int x = 1 << (poly_power_depth(k) - 1), y = k - x;
        p->tree.push_back({k, x, y});
        const int l = std::min(lv[x], lv[y]);
        p->pw_scale[k] = (p->pw_scale[x] * p->pw_scale[y]) / (double)c->primes[l];
        lv[k] = l - 1;
    }
    p->level_c = level - poly_power_depth(d);
    const double qc = (double)c->primes[p->level_c];
    for (int k = 1; k <= d; k++) {
        if (a[k] == 0.0) continue;
        const double s = (target * qc) / p->pw_scale[k];
        const double v = round_half_away(a[k] * s);
        HCHECK(std::isfinite(v), HELRM_E_PARAM, "polynomial coefficient too large for the scale");
        ActPlan::Term t;
        t.k = k;
        t.scale = p->pw_scale[k] * s;
        t.mont = int_table_f(c, v, true);
        p->terms.push_back(std::move(t));
    }
    HCHECK(!p->terms.empty(), HELRM_E_INVAL, "need a non-constant polynomial");
    p->out_level = p->level_c - 1;
    p->out_scale = p->terms[0].scale / qc;
    if (a[0] != 0.0) {
        const double v = round_half_away(a[0] * p->out_scale);
        HCHECK(std::isfinite(v), HELRM_E_PARAM, "constant term too large for the scale");
        p->a0 = int_table_f(c, v, false);
    }
    return p.release();
}

Ciphertext *ct_poly_eval(Ctx *c, const EvalKey *evk, const Ciphertext *x, const std::vector<double> &a, double target)
{
    std::unique_ptr<ActPlan> plan(act_plan(c, a, x->level, x->scale, target));
    std::vector<Ciphertext *> y = poly_b(c, {evk}, {x}, *plan);
    return y[0];
}

}  // namespace helrm
