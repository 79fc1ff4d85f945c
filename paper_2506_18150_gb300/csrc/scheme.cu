// scheme.cu -- RNS-CKKS on the device (HE-LRM appendix "CKKS operations").
//
// Keys: ternary secret s (CBD(1)), public key (-a s + e, a), and hybrid
// key-switching keys: for digit j (primes [j alpha, (j+1) alpha) of Q), over
// every limb of QP, b_j = -a_j s + e_j + [P]_{q_i} s' on the digit's primes and
// b_j = -a_j s + e_j elsewhere; s' = s^2 (relinearisation) or phi_k(s) (rotation).
// a is uniform mod q (drawn in the coefficient domain), e is CBD(21); every
// value comes from a ChaCha20 stream (seed, purpose, index).
//
// Key switching at level l: ModUp (iNTT, fast base conversion of each digit to
// all other limbs of QP_l, NTT), the inner product with the key, ModDown
// (out = (u - FBC_{P->Q}([u]_P)) P^-1, no rounding offset).  Rotation applies
// the Galois map to the extended digits (ModUp first, then phi), as hoisting
// requires.  Rescale subtracts the centred remainder of the dropped limb and
// multiplies by q_l^-1, which is round(x / q_l).
#include <cstring>

#include "core.cuh"

namespace helrm {

enum Purpose : u32 { P_SK = 1, P_PK_A, P_PK_E, P_KSK_A, P_KSK_E, P_ENC_V, P_ENC_E0, P_ENC_E1, P_SK_SPARSE };

Ciphertext *new_ct(Ctx *c, int level, double scale)
{
    std::unique_ptr<Ciphertext> ct(new Ciphertext(c));
    ct->level = level;
    ct->scale = scale;
    ct->data = DevMem(c, (size_t)2 * (level + 1) * c->N * 8);
    return ct.release();
}

// ---------------------------------------------------------------- ModUp / ModDown
// The fast base conversion runs inside the two transforms around it: the
// inverse NTT of a source limb ends with N^-1 [(Q_j/q_s)^-1]_{q_s} instead of
// N^-1, and the forward NTT of each converted limb computes its input from
// the digit's source limbs on load (NttLimb::scal / fbc_*).
void modup_limbs(Ctx *c, int level, const u64 *poly, u64 *coef, u64 *digits, std::vector<k::NttLimb> &inv,
                 std::vector<k::NttLimb> &fwd)
{
    const int N = c->N, nl = level + 1 + c->K;
    const LimbMap m = c->qmap(level);
    for (int j = 0; j < c->dnum(level); j++) {
        const BConvTable &t = c->modup_table(level, j);
        const int lo = c->digit_lo(j), hi = c->digit_hi(j, level);
        for (int l = lo; l < hi; l++) {
            k::NttLimb x{poly + (size_t)l * N, coef + (size_t)l * N, m.pid(l), nullptr, nullptr, nullptr};
            x.scal = t.scale(l - lo);
            inv.push_back(x);
        }
        int kd = 0;   // destinations in limb order: every limb outside the digit
        for (int l = 0; l < nl; l++) {
            if (l >= lo && l < hi) continue;
            k::NttLimb x{coef + (size_t)lo * N, digits + ((size_t)j * nl + l) * N, m.pid(l), nullptr, nullptr, nullptr};
            x.fbc_n = hi - lo;
            x.fbc_h = t.hcol(kd++);
            x.fbc_hs = t.n_dst;
            fwd.push_back(x);
        }
    }
}

void ks_modup(Ctx *c, const u64 *poly, int level, u64 *digits)
{
    const int N = c->N, nq = level + 1, nl = nq + c->K;
    DevMem coef(c, (size_t)nq * N * 8);
    std::vector<k::NttLimb> inv, fwd;
    modup_limbs(c, level, poly, coef.u(), digits, inv, fwd);
    k::ntt_run(c, inv, true, nullptr);
    for (int j = 0; j < c->dnum(level); j++) {   // each digit keeps its own limbs as they are
        const int lo = c->digit_lo(j), hi = c->digit_hi(j, level);
        k::copy(c, digits + ((size_t)j * nl + lo) * N, poly + (size_t)lo * N, (size_t)(hi - lo) * N);
    }
    k::ntt_run(c, fwd, false, nullptr);
}

// ModDown of both halves of a QP ciphertext u = [2][nl][N] into out0, out1.
// The iNTT reads the P limbs of u in place of a copy; the forward NTT of the
// converted limbs ends with out = (u - y) * P^-1 (+ add) fused into its last pass.
// One half of a ModDown: the iNTT of the K P-limbs of qp (into pc, scaled by
// N^-1 [(P/p_i)^-1]_{p_i}) and the forward NTT of each Q-limb l converted
// from them on load (through y), ending with out = (qp_l - y) P^-1 (+ add).
void moddown_limbs(Ctx *c, int level, const u64 *qp, u64 *pc, u64 *y, u64 *out, const u64 *add,
                   std::vector<k::NttLimb> &inv, std::vector<k::NttLimb> &fwd)
{
    const int N = c->N, nq = level + 1, K = c->K;
    const LimbMap m = c->qmap(level);
    const BConvTable &t = c->moddown_table(level);
    for (int i = 0; i < K; i++) {
        k::NttLimb x{qp + (size_t)(nq + i) * N, pc + (size_t)i * N, m.pid(nq + i), nullptr, nullptr, nullptr};
        x.scal = t.scale(i);
        inv.push_back(x);
    }
    for (int l = 0; l < nq; l++) {
        k::NttLimb x{pc, y + (size_t)l * N, m.pid(l), qp + (size_t)l * N, out + (size_t)l * N,
                     add ? add + (size_t)l * N : nullptr};
        x.fbc_n = K;
        x.fbc_h = t.hcol(l);
        x.fbc_hs = t.n_dst;
        fwd.push_back(x);
    }
}

void ks_moddown2(Ctx *c, const u64 *u, int level, u64 *out0, u64 *out1, const u64 *add0, const u64 *add1)
{
    const int N = c->N, nq = level + 1, K = c->K, nl = nq + K;
    DevMem pc(c, (size_t)2 * K * N * 8), y(c, (size_t)2 * nq * N * 8);
    std::vector<k::NttLimb> inv, fwd;
    for (int h = 0; h < 2; h++)
        moddown_limbs(c, level, u + (size_t)h * nl * N, pc.u() + (size_t)h * K * N, y.u() + (size_t)h * nq * N,
                      h ? out1 : out0, h ? add1 : add0, inv, fwd);
    k::ntt_run(c, inv, true, nullptr);
    k::ntt_run(c, fwd, false, c->d_pinv_mont.u());
}

void ks_moddown(Ctx *c, const u64 *u, int level, u64 *out)
{
    const int N = c->N, nq = level + 1, K = c->K;
    DevMem pc(c, (size_t)K * N * 8), y(c, (size_t)nq * N * 8);
    std::vector<k::NttLimb> inv, fwd;
    moddown_limbs(c, level, u, pc.u(), y.u(), out, nullptr, inv, fwd);
    k::ntt_run(c, inv, true, nullptr);
    k::ntt_run(c, fwd, false, c->d_pinv_mont.u());
}

const SwitchKey *rot_key(const EvalKey *evk, u64 galois, int level)
{
    auto it = evk->rot.find(galois);
    HCHECK(it != evk->rot.end(), HELRM_E_NOKEY, "no rotation key for galois element " + std::to_string(galois));
    HCHECK(it->second->level >= level, HELRM_E_NOKEY,
           "the rotation key for galois element " + std::to_string(galois) + " was generated up to level " +
               std::to_string(it->second->level) + ", below its use at level " + std::to_string(level));
    return it->second.get();
}

const SwitchKey *relin_key(const EvalKey *evk, int level)
{
    HCHECK(evk->relin, HELRM_E_NOKEY, "no relinearisation key");
    HCHECK(evk->relin->level >= level, HELRM_E_NOKEY, "the relinearisation key was generated below its use");
    return evk->relin.get();
}

// ---------------------------------------------------------------- basic ops
static void check_pair(const Ciphertext *a, const Ciphertext *b)
{
    HCHECK(a->level == b->level, HELRM_E_LEVEL, "ciphertext levels differ");
    HCHECK(std::fabs(a->scale - b->scale) <= 1e-9 * a->scale, HELRM_E_SCALE, "ciphertext scales differ");
}

Ciphertext *ct_add(Ctx *c, const Ciphertext *a, const Ciphertext *b, bool subtract)
{
    check_pair(a, b);
    std::unique_ptr<Ciphertext> o(new_ct(c, a->level, a->scale));
    int n = 2 * (a->level + 1);
    if (subtract)
        k::sub(c, o->data.u(), a->data.u(), b->data.u(), n, c->qmap(a->level, 0, a->level + 1));
    else
        k::add(c, o->data.u(), a->data.u(), b->data.u(), n, c->qmap(a->level, 0, a->level + 1));
    return o.release();
}

Ciphertext *ct_add_pt(Ctx *c, const Ciphertext *a, const Plaintext *pt)
{
    HCHECK(pt->form == PT_PLAIN, HELRM_E_INVAL, "plaintext is in multiplier form");
    HCHECK(pt->level >= a->level, HELRM_E_LEVEL, "plaintext level below ciphertext level");
    HCHECK(std::fabs(a->scale - pt->scale) <= 1e-9 * a->scale, HELRM_E_SCALE, "plaintext scale differs");
    std::unique_ptr<Ciphertext> o(new_ct(c, a->level, a->scale));
    const int nq = a->level + 1;
    k::add(c, o->c0(), a->c0(), pt->data.u(), nq, c->qmap(a->level));
    k::copy(c, o->c1(), a->c1(), (size_t)nq * c->N);
    return o.release();
}

Ciphertext *ct_mul_pt(Ctx *c, const Ciphertext *a, const Plaintext *pt)
{
    HCHECK(pt->level >= a->level && !pt->qp, HELRM_E_LEVEL, "plaintext level below ciphertext level");
    std::unique_ptr<Ciphertext> o(new_ct(c, a->level, a->scale * pt->scale));
    const int nq = a->level + 1;
    for (int p = 0; p < 2; p++) {
        u64 *dst = p ? o->c1() : o->c0();
        const u64 *src = p ? a->c1() : a->c0();
        if (pt->form == PT_MONT)
            k::mul_mont(c, dst, src, pt->data.u(), nq, c->qmap(a->level));
        else
            k::mul_plain(c, dst, src, pt->data.u(), nq, c->qmap(a->level));
    }
    return o.release();
}

Ciphertext *ct_drop(Ctx *c, const Ciphertext *a, int level)
{
    HCHECK(level >= 0 && level <= a->level, HELRM_E_LEVEL, "cannot raise the level");
    std::unique_ptr<Ciphertext> o(new_ct(c, level, a->scale));
    k::copy(c, o->c0(), a->c0(), (size_t)(level + 1) * c->N);
    k::copy(c, o->c1(), a->c1(), (size_t)(level + 1) * c->N);
    return o.release();
}

Ciphertext *ct_rescale(Ctx *c, const Ciphertext *a)
{
    const int l = a->level, N = c->N;
    HCHECK(l >= 1, HELRM_E_LEVEL, "no level left to rescale");
    std::unique_ptr<Ciphertext> o(new_ct(c, l - 1, a->scale / (double)c->primes[l]));
    DevMem last(c, (size_t)2 * N * 8), r(c, (size_t)2 * l * N * 8);
    std::vector<k::NttLimb> v = {{a->c0() + (size_t)l * N, last.u(), l, nullptr, nullptr},
                                 {a->c1() + (size_t)l * N, last.u() + N, l, nullptr, nullptr}};
    k::ntt_run(c, v, true, nullptr);
    k::rescale_spread(c, r.u(), last.u(), l, 2);
    // out = (a - r) * q_l^-1, fused into the last pass of the forward NTT of r
    v.clear();
    for (int h = 0; h < 2; h++)
        for (int i = 0; i < l; i++) {
            u64 *ri = r.u() + (size_t)(h * l + i) * N;
            v.push_back({ri, ri, i, (h ? a->c1() : a->c0()) + (size_t)i * N, (h ? o->c1() : o->c0()) + (size_t)i * N});
        }
    k::ntt_run(c, v, false, c->rescale_table(l));
    return o.release();
}

// ---------------------------------------------------------------- rotation
void ct_rotate_hoisted(Ctx *c, const EvalKey *evk, const Ciphertext *a, const std::vector<int> &steps,
                       std::vector<Ciphertext *> &outs)
{
    const int l = a->level, N = c->N, nq = l + 1, nl = nq + c->K, dnum = c->dnum(l);
    std::vector<std::unique_ptr<Ciphertext>> res;
    std::vector<const SwitchKey *> keys;
    for (int st : steps) keys.push_back(c->galois(st) == 1 ? nullptr : rot_key(evk, c->galois(st), l));
    DevMem digits(c, (size_t)dnum * nl * N * 8), u(c, (size_t)2 * nl * N * 8);
    ks_modup(c, a->c1(), l, digits.u());
    for (size_t s = 0; s < steps.size(); s++) {
        u64 g = c->galois(steps[s]);
        std::unique_ptr<Ciphertext> o(new_ct(c, l, a->scale));
        if (g == 1) {
            k::copy(c, o->data.u(), a->data.u(), (size_t)2 * nq * N);
        } else {
            k::ks_inner_auto(c, u.u(), digits.u(), dnum, keys[s], l, g, nullptr, nullptr);
            k::automorphism(c, o->c0(), a->c0(), nq, g);
            ks_moddown2(c, u.u(), l, o->c0(), o->c1(), o->c0());   // phi(c0) + ModDown(u_0)
        }
        res.push_back(std::move(o));
    }
    outs.clear();
    for (auto &r : res) outs.push_back(r.release());
}

// X -> X^g with the key switch, in a hoisted rotation's order (ModUp of c1,
// then phi_g on the extended digits inside the key inner product)
Ciphertext *ct_apply_galois(Ctx *c, const EvalKey *evk, const Ciphertext *a, u64 g)
{
    const int l = a->level, N = c->N, nq = l + 1, nl = nq + c->K, dnum = c->dnum(l);
    const SwitchKey *key = rot_key(evk, g, l);
    DevMem digits(c, (size_t)dnum * nl * N * 8), u(c, (size_t)2 * nl * N * 8);
    ks_modup(c, a->c1(), l, digits.u());
    std::unique_ptr<Ciphertext> o(new_ct(c, l, a->scale));
    k::ks_inner_auto(c, u.u(), digits.u(), dnum, key, l, g, nullptr, nullptr);
    k::automorphism(c, o->c0(), a->c0(), nq, g);
    ks_moddown2(c, u.u(), l, o->c0(), o->c1(), o->c0());
    return o.release();
}

Ciphertext *ct_rotate(Ctx *c, const EvalKey *evk, const Ciphertext *a, int step)
{
    std::vector<Ciphertext *> outs;
    ct_rotate_hoisted(c, evk, a, {step}, outs);
    return outs[0];
}

// ---------------------------------------------------------------- ct x ct
void ct_tensor_acc(Ctx *c, u64 *d012, const Ciphertext *a, const Ciphertext *b, bool accumulate)
{
    HCHECK(a->level == b->level, HELRM_E_LEVEL, "ciphertext levels differ");
    k::tensor(c, d012, a->c0(), a->c1(), b->c0(), b->c1(), a->level + 1, c->qmap(a->level), accumulate);
}

Ciphertext *ct_relin(Ctx *c, const EvalKey *evk, const u64 *d012, int level, double scale)
{
    const SwitchKey *rk = relin_key(evk, level);
    const int N = c->N, nq = level + 1, nl = nq + c->K, dnum = c->dnum(level);
    const size_t plane = (size_t)nq * N;
    DevMem digits(c, (size_t)dnum * nl * N * 8), u(c, (size_t)2 * nl * N * 8);
    ks_modup(c, d012 + 2 * plane, level, digits.u());
    k::ks_inner_auto(c, u.u(), digits.u(), dnum, rk, level, 1, nullptr, nullptr);
    std::unique_ptr<Ciphertext> o(new_ct(c, level, scale));
    ks_moddown2(c, u.u(), level, o->c0(), o->c1(), d012, d012 + plane);   // (d0, d1) + ModDown(u)
    return o.release();
}

Ciphertext *ct_mul(Ctx *c, const EvalKey *evk, const Ciphertext *a, const Ciphertext *b)
{
    HCHECK(a->level == b->level, HELRM_E_LEVEL, "ciphertext levels differ");
    HCHECK(a->level >= 1, HELRM_E_LEVEL, "no level left for a multiplication");
    DevMem d(c, (size_t)3 * (a->level + 1) * c->N * 8);
    ct_tensor_acc(c, d.u(), a, b, false);
    std::unique_ptr<Ciphertext> r(ct_relin(c, evk, d.u(), a->level, a->scale * b->scale));
    return ct_rescale(c, r.get());
}

// ---------------------------------------------------------------- plaintexts
Plaintext *pt_encode(Ctx *c, const double *h_slots, int n_slots, int period, int level, bool qp, double scale,
                     int form, const double *h_slots_im)
{
    HCHECK(level >= 0 && level <= c->L, HELRM_E_LEVEL, "level out of range");
    HCHECK(period >= 1 && period <= c->n_slots && (c->n_slots % period) == 0 && n_slots <= period,
           HELRM_E_INVAL, "slot period must divide n and hold the values");
    std::unique_ptr<Plaintext> pt(new Plaintext(c));
    pt->level = level;
    pt->qp = qp;
    pt->form = form;
    pt->scale = scale;
    const int nl = pt->limbs();
    pt->data = DevMem(c, (size_t)nl * c->N * 8);
    DevMem ds(c, (size_t)std::max(n_slots, 1) * 8 * (h_slots_im ? 2 : 1));
    if (n_slots) CUDA_CHECK(cudaMemcpyAsync(ds.ptr, h_slots, (size_t)n_slots * 8, cudaMemcpyHostToDevice, c->stream));
    if (n_slots && h_slots_im)
        CUDA_CHECK(cudaMemcpyAsync(ds.as<double>() + n_slots, h_slots_im, (size_t)n_slots * 8,
                                   cudaMemcpyHostToDevice, c->stream));
    k::encode_slots(c, pt->data.u(), ds.as<double>(), n_slots, period, scale, nl, c->qmap(level), nullptr,
                    h_slots_im ? ds.as<double>() + n_slots : nullptr);
    k::ntt_fwd(c, pt->data.u(), nl, c->qmap(level));
    if (form == PT_MONT) k::to_mont(c, pt->data.u(), pt->data.u(), nl, c->qmap(level));
    return pt.release();
}

Plaintext *pt_encode_dev(Ctx *c, const double *d_slots, int n_valid, int period, int level, double scale)
{
    HCHECK(period >= 1 && period <= c->n_slots && (c->n_slots % period) == 0 && n_valid <= period, HELRM_E_INVAL,
           "slot period must divide n and hold the values");
    std::unique_ptr<Plaintext> pt(new Plaintext(c));
    pt->level = level;
    pt->scale = scale;
    const int nl = pt->limbs();
    pt->data = DevMem(c, (size_t)nl * c->N * 8);
    k::encode_slots(c, pt->data.u(), d_slots, n_valid, period, scale, nl, c->qmap(level), nullptr);
    k::ntt_fwd(c, pt->data.u(), nl, c->qmap(level));
    return pt.release();
}

Plaintext *pt_from_signed(Ctx *c, const i64 *h_coeffs, int level, bool qp, double scale, int form)
{
    HCHECK(level >= 0 && level <= c->L, HELRM_E_LEVEL, "level out of range");
    std::unique_ptr<Plaintext> pt(new Plaintext(c));
    pt->level = level;
    pt->qp = qp;
    pt->form = form;
    pt->scale = scale;
    const int nl = pt->limbs();
    pt->data = DevMem(c, (size_t)nl * c->N * 8);
    DevMem ds(c, (size_t)c->N * 8);
    CUDA_CHECK(cudaMemcpyAsync(ds.ptr, h_coeffs, (size_t)c->N * 8, cudaMemcpyHostToDevice, c->stream));
    k::from_signed(c, pt->data.u(), ds.as<i64>(), nl, c->qmap(level));
    k::ntt_fwd(c, pt->data.u(), nl, c->qmap(level));
    if (form == PT_MONT) k::to_mont(c, pt->data.u(), pt->data.u(), nl, c->qmap(level));
    return pt.release();
}

void pt_export_signed(Ctx *c, const Plaintext *pt, i64 *h_out)
{
    const int N = c->N;
    DevMem t(c, (size_t)N * 8);
    if (pt->form == PT_MONT)
        k::from_mont(c, t.u(), pt->data.u(), 1, c->qmap(0));
    else
        k::copy(c, t.u(), pt->data.u(), N);
    k::ntt_inv(c, t.u(), 1, c->qmap(0));
    std::vector<u64> h(N);
    CUDA_CHECK(cudaMemcpyAsync(h.data(), t.ptr, (size_t)N * 8, cudaMemcpyDeviceToHost, c->stream));
    c->check_device_errors();
    const u64 q0 = c->primes[0];
    for (int i = 0; i < N; i++) h_out[i] = h[i] > (q0 - 1) / 2 ? -(i64)(q0 - h[i]) : (i64)h[i];
}

// ---------------------------------------------------------------- keys
struct LimbIds {   // device arrays: prime id and global QP position of each limb
    DevMem pid, gid;
};
// the limbs q_0..q_kl, p_0..p_{K-1} (global prime ids, which are also their QP positions)
static LimbIds level_limbs(Ctx *c, int kl)
{
    const int n = kl + 1 + c->K;
    std::vector<int> ids(n);
    for (int i = 0; i < n; i++) ids[i] = c->qmap(kl).pid(i);
    LimbIds r;
    r.pid = DevMem(c, n * 4);
    r.gid = DevMem(c, n * 4);
    CUDA_CHECK(cudaMemcpyAsync(r.pid.ptr, ids.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(r.gid.ptr, ids.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    return r;
}
static LimbIds full_limbs(Ctx *c, int n)
{
    HCHECK(n == c->nP(), HELRM_E_PARAM, "internal: full limb list");
    return level_limbs(c, c->L);
}

SecretKey *keygen_sk(Ctx *c, u64 seed, int h)
{
    std::unique_ptr<SecretKey> sk(new SecretKey(c));
    const int nP = c->nP(), N = c->N;
    LimbMap all = c->qmap(c->L);
    DevMem s(c, (size_t)N * 8);
    if (h > 0)
        k::sample_sparse_ternary(c, s.as<i64>(), seed, P_SK_SPARSE, h);
    else
        k::sample_ternary(c, s.as<i64>(), seed, P_SK, 0);
    sk->s_ntt = DevMem(c, (size_t)nP * N * 8);
    sk->s_mont = DevMem(c, (size_t)nP * N * 8);
    k::from_signed(c, sk->s_ntt.u(), s.as<i64>(), nP, all);
    k::ntt_fwd(c, sk->s_ntt.u(), nP, all);
    k::to_mont(c, sk->s_mont.u(), sk->s_ntt.u(), nP, all);
    return sk.release();
}

// b = -a s + e (+ [P]_{q_i} s' on digit j's primes) over the limbs q_0..q_kl,
// p_0..p_{K-1} of a key of level kl; stored (b, a) in Montgomery form at `out`.
// Every sample is addressed by its global QP position, so a key of level kl is
// exactly the restriction of the full (kl = L) key.
static void make_switch_digit(Ctx *c, const SecretKey *sk, u64 seed, u64 index, const u64 *s_prime, int j, int kl,
                              const LimbIds &ids, u64 *out)
{
    const int N = c->N, nq = kl + 1, nK = nq + c->K;
    const size_t plane = (size_t)nK * N;
    const LimbMap km = c->qmap(kl);
    u64 *b = out, *a = out + plane;
    DevMem e(c, (size_t)N * 8), t(c, plane * 8);
    k::sample_uniform(c, a, seed, P_KSK_A, index, nK, ids.pid.as<int>(), ids.gid.as<int>());
    k::ntt_fwd(c, a, nK, km);
    k::sample_cbd21(c, e.as<i64>(), seed, P_KSK_E, index);
    k::from_signed(c, b, e.as<i64>(), nK, km);
    k::ntt_fwd(c, b, nK, km);
    // a s: s over the Q limbs 0..kl, then over the P limbs (stored after q_L)
    k::mul_mont(c, t.u(), a, sk->s_mont.u(), nq, km);
    k::mul_mont(c, t.u() + (size_t)nq * N, a + (size_t)nq * N, sk->s_mont.u() + (size_t)(c->L + 1) * N, c->K,
                c->qmap(kl, nq));
    k::sub(c, b, b, t.u(), nK, km);
    if (s_prime) {
        const int lo = c->digit_lo(j), hi = c->digit_hi(j, kl);
        k::mul_scalar_mont(c, t.u(), s_prime + (size_t)lo * N, c->d_pmod_mont.u(), hi - lo, c->qmap(kl, lo));
        k::add(c, b + (size_t)lo * N, b + (size_t)lo * N, t.u(), hi - lo, c->qmap(kl, lo));
    }
    k::to_mont(c, out, out, 2 * nK, c->qmap(kl, 0, nK));
}

static std::unique_ptr<SwitchKey> make_switch_key(Ctx *c, const SecretKey *sk, u64 seed, u64 key_id,
                                                  const u64 *s_prime, int kl, const LimbIds &ids)
{
    std::unique_ptr<SwitchKey> key(new SwitchKey());
    key->level = kl;
    key->dnum = c->dnum(kl);
    const size_t per = (size_t)2 * (kl + 1 + c->K) * c->N;
    key->data = DevMem(c, key->dnum * per * 8);
    for (int j = 0; j < key->dnum; j++)
        make_switch_digit(c, sk, seed, (key_id << 8) | (u64)j, s_prime, j, kl, ids, key->data.u() + j * per);
    return key;
}

EvalKey *keygen_evk(Ctx *c, const SecretKey *sk, u64 seed, int relin_level)
{
    if (relin_level < 0) relin_level = c->L;
    HCHECK(relin_level <= c->L, HELRM_E_LEVEL, "key level above the chain");
    std::unique_ptr<EvalKey> evk(new EvalKey(c));
    evk->seed = seed;
    const int nq = c->L + 1, nP = c->nP(), N = c->N;
    LimbIds ids = full_limbs(c, nP);
    LimbMap qm = c->qmap(c->L);
    // public key over q_0..q_L
    evk->pk = DevMem(c, (size_t)2 * nq * N * 8);
    u64 *b = evk->pk.u(), *a = evk->pk.u() + (size_t)nq * N;
    DevMem e(c, (size_t)N * 8), t(c, (size_t)nq * N * 8);
    k::sample_uniform(c, a, seed, P_PK_A, 0, nq, ids.pid.as<int>(), ids.gid.as<int>());
    k::ntt_fwd(c, a, nq, qm);
    k::sample_cbd21(c, e.as<i64>(), seed, P_PK_E, 0);
    k::from_signed(c, b, e.as<i64>(), nq, qm);
    k::ntt_fwd(c, b, nq, qm);
    k::mul_mont(c, t.u(), a, sk->s_mont.u(), nq, qm);
    k::sub(c, b, b, t.u(), nq, qm);
    k::to_mont(c, evk->pk.u(), evk->pk.u(), 2 * nq, c->qmap(c->L, 0, nq));
    // relinearisation key: s' = s^2
    DevMem s2(c, (size_t)nP * N * 8);
    k::mul_mont(c, s2.u(), sk->s_ntt.u(), sk->s_mont.u(), nP, c->qmap(c->L));
    LimbIds rids = level_limbs(c, relin_level);
    evk->relin = make_switch_key(c, sk, seed, 0, s2.u(), relin_level, rids);
    return evk.release();
}

void keygen_rot(Ctx *c, const SecretKey *sk, EvalKey *evk, const std::vector<int> &steps,
                const std::vector<int> &levels)
{
    std::vector<u64> gals;
    for (int st : steps) gals.push_back(c->galois(st));
    keygen_galois(c, sk, evk, gals, levels);
}

void keygen_galois(Ctx *c, const SecretKey *sk, EvalKey *evk, const std::vector<u64> &gals,
                   const std::vector<int> &levels)
{
    const int nP = c->nP(), N = c->N;
    std::map<int, LimbIds> ids;
    DevMem sp(c, (size_t)nP * N * 8);
    for (size_t i = 0; i < gals.size(); i++) {
        const u64 g = gals[i];
        HCHECK((g & 1) && g < 2ull * N, HELRM_E_INVAL, "a Galois element is odd and below 2N");
        const int kl = levels.empty() ? c->L : levels[i];
        HCHECK(kl >= 0 && kl <= c->L, HELRM_E_LEVEL, "key level outside the chain");
        if (g == 1) continue;
        auto it = evk->rot.find(g);
        if (it != evk->rot.end() && it->second->level >= kl) continue;
        if (!ids.count(kl)) ids[kl] = level_limbs(c, kl);
        k::automorphism(c, sp.u(), sk->s_ntt.u(), nP, g);   // phi_g(s), NTT domain
        evk->rot[g] = make_switch_key(c, sk, evk->seed, g, sp.u(), kl, ids[kl]);
    }
}

// ---------------------------------------------------------------- enc / dec
Ciphertext *encrypt_pt(Ctx *c, const EvalKey *evk, const Plaintext *pt, u64 seed)
{
    HCHECK(pt->form == PT_PLAIN && !pt->qp, HELRM_E_INVAL, "plaintext must be a plain Q-basis plaintext");
    const int l = pt->level, nq = l + 1, N = c->N, nqL = c->L + 1;
    std::unique_ptr<Ciphertext> ct(new_ct(c, l, pt->scale));
    LimbMap qm = c->qmap(l);
    // v, e0 and e1 (each sampled from its own counter stream) are transformed
    // by one NTT launch: vee = [v | e0 | e1], each nq limbs
    DevMem raw(c, (size_t)3 * N * 8), vee(c, (size_t)3 * nq * N * 8);
    k::sample_enc_noise(c, raw.as<i64>(), seed, P_ENC_V, P_ENC_E0, P_ENC_E1);
    k::from_signed(c, vee.u(), raw.as<i64>(), nq, qm, 3);
    k::ntt_fwd(c, vee.u(), 3 * nq, c->qmap(l, 0, nq));
    const size_t pl = (size_t)nq * N;
    k::enc_combine(c, ct->c0(), ct->c1(), vee.u(), vee.u() + pl, vee.u() + 2 * pl, pt->data.u(), evk->pk.u(),
                   evk->pk.u() + (size_t)nqL * N, nq, qm);
    return ct.release();
}

void decrypt_slots_device(Ctx *c, const SecretKey *sk, const Ciphertext *ct, double *d_out, int n_slots)
{
    HCHECK(n_slots >= 1 && n_slots <= c->n_slots, HELRM_E_INVAL, "n_slots out of range");
    DevMem m(c, (size_t)c->N * 8);
    k::mul_mont(c, m.u(), ct->c1(), sk->s_mont.u(), 1, c->qmap(0));
    k::add(c, m.u(), m.u(), ct->c0(), 1, c->qmap(0));
    k::ntt_inv(c, m.u(), 1, c->qmap(0));
    k::decode_limb0(c, d_out, m.u(), ct->scale, n_slots);
}

void decrypt_slots(Ctx *c, const SecretKey *sk, const Ciphertext *ct, double *h_out, int n_slots)
{
    HCHECK(n_slots >= 0 && n_slots <= c->n_slots, HELRM_E_INVAL, "n_slots out of range");
    const int N = c->N;
    DevMem m(c, (size_t)N * 8), d(c, (size_t)std::max(n_slots, 1) * 8);
    k::mul_mont(c, m.u(), ct->c1(), sk->s_mont.u(), 1, c->qmap(0));
    k::add(c, m.u(), m.u(), ct->c0(), 1, c->qmap(0));
    k::ntt_inv(c, m.u(), 1, c->qmap(0));
    if (n_slots) {
        k::decode_limb0(c, d.as<double>(), m.u(), ct->scale, n_slots);
        CUDA_CHECK(cudaMemcpyAsync(h_out, d.ptr, (size_t)n_slots * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    c->check_device_errors();
}

}  // namespace helrm
