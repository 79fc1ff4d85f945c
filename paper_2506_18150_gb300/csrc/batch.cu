// batch.cu -- lockstep batched inference: B queries of one model, each with
// its own client's evaluation keys, advance through the layers together, and
// every step of the path is one launch for the whole batch.
//
// Nothing in the arithmetic changes: each query goes through exactly the
// integer operations of the op-by-op CKKS primitives (linear.cu matvec,
// scheme.cu rotations, products, rescale), so its logit ciphertext does not
// depend on what it is batched with.  One query alone (helrm_infer) is a
// batch of one.  What changes is the launch shape:
//  * NTTs, base conversions, key inner products, automorphisms and
//    elementwise ops take job lists covering every query (and, where the
//    steps are independent, every giant step or rotation as well);
//  * the fused baby-step + BSGS kernel runs all queries in one grid whose
//    fastest index is the query, so the CTAs that share a diagonal tile run
//    together and the diagonal rows are fetched from HBM once per batch
//    instead of once per query (the weight diagonals are the same for every
//    client; the keys are not);
//  * the per-query key tables of every matrix are built once, when the batch
//    is created, so a batch can be replayed as a CUDA graph
//    (model_infer_batch_graph, below).
#include <cmath>

#include "model.cuh"

namespace helrm {
namespace {

constexpr int BJ = 256;   // jobs per batched launch (kernel-parameter arrays)
constexpr int TPB = 256;

inline unsigned gx_for(size_t total, int n_jobs)
{
    size_t g = (total + TPB - 1) / TPB;
    size_t cap = std::max<size_t>(4, (size_t)152 * 32 / std::max(1, n_jobs));
    return (unsigned)std::min(g, cap);
}

enum BOp { B_ADD, B_SUB, B_MULM, B_MULP };

struct EwJobs {
    int n;
    u64 *o[BJ];
    const u64 *a[BJ];
    const u64 *b[BJ];
};

__global__ void k_ew_b(const EwJobs J, int logN, size_t total, const PrimeInfo *__restrict__ pinfo, LimbMap map,
                       int op)
{
    pdl_begin();
    u64 *__restrict__ o = J.o[blockIdx.y];
    const u64 *__restrict__ a = J.a[blockIdx.y];
    const u64 *__restrict__ b = J.b[blockIdx.y];
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const PrimeInfo pi = pinfo[map.pid((int)(idx >> logN))];
        const u64 x = a[idx];
        u64 r;
        switch (op) {
        case B_ADD: r = add_mod(x, b[idx], pi.q); break;
        case B_SUB: r = sub_mod(x, b[idx], pi.q); break;
        case B_MULM: r = mont_mul(x, b[idx], pi.q, pi.qinv); break;
        default: r = mul_mod(x, b[idx], pi.q, pi.qinv, pi.r2); break;
        }
        o[idx] = r;
    }
}

struct CopyJobs {
    int n;
    u64 *o[BJ];
    const u64 *a[BJ];
    u64 words[BJ];
};

__global__ void k_copy_b(const CopyJobs J)
{
    pdl_begin();
    const uint2 *__restrict__ a = (const uint2 *)J.a[blockIdx.y];
    uint2 *__restrict__ o = (uint2 *)J.o[blockIdx.y];
    const u64 n = J.words[blockIdx.y];
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) o[i] = a[i];
}

struct TensorJobs {
    int n;
    u64 *d[BJ];
    const u64 *a0[BJ];
    const u64 *a1[BJ];
    const u64 *b0[BJ];
    const u64 *b1[BJ];
};

// (d0, d1, d2) (+)= (a0 b0, a0 b1 + a1 b0, a1 b1), as k_tensor
__global__ void k_tensor_b(const TensorJobs J, int logN, size_t total, const PrimeInfo *__restrict__ pinfo,
                           LimbMap map, int accumulate)
{
    pdl_begin();
    const int j = blockIdx.y;
    u64 *__restrict__ d = J.d[j];
    const u64 *__restrict__ a0 = J.a0[j];
    const u64 *__restrict__ a1 = J.a1[j];
    const u64 *__restrict__ b0 = J.b0[j];
    const u64 *__restrict__ b1 = J.b1[j];
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const PrimeInfo pi = pinfo[map.pid((int)(idx >> logN))];
        const u64 x0 = a0[idx], x1 = a1[idx], y0 = b0[idx], y1 = b1[idx];
        Acc128 s0, s1, s2;
        s0.mac(x0, y0, pi.q);
        s1.mac(x0, y1, pi.q);
        s1.mac(x1, y0, pi.q);
        s2.mac(x1, y1, pi.q);
        u64 r0 = mont_mul(s0.reduce(pi.q, pi.qinv), pi.r2, pi.q, pi.qinv);
        u64 r1 = mont_mul(s1.reduce(pi.q, pi.qinv), pi.r2, pi.q, pi.qinv);
        u64 r2 = mont_mul(s2.reduce(pi.q, pi.qinv), pi.r2, pi.q, pi.qinv);
        if (accumulate) {
            r0 = add_mod(r0, d[idx], pi.q);
            r1 = add_mod(r1, d[total + idx], pi.q);
            r2 = add_mod(r2, d[2 * total + idx], pi.q);
        }
        d[idx] = r0;
        d[total + idx] = r1;
        d[2 * total + idx] = r2;
    }
}

__device__ __forceinline__ int auto_src_b(int i, int logN, u64 galois)
{
    const u32 x = __brev((u32)i) >> (32 - logN);
    const u64 e = ((2ull * x + 1) * galois) & ((2ull << logN) - 1);
    return (int)(__brev((u32)((e - 1) >> 1)) >> (32 - logN));
}

struct KsJobs {
    int n;
    u64 *out[BJ];
    const u64 *dig[BJ];
    const u64 *key[BJ];
    const u64 *c0[BJ];
    const u64 *bq[BJ];
    u64 gal[BJ];
    int kl[BJ];           // level the job's key was generated up to
};

// Fused automorphism + key inner product of k_ks_inner, one job per
// (query, key): out_h[l][i] = sum_j dig_j[l][src(i)] key_j,h[pid(l)][i]
// (+ P c0[l][src(i)] on the Q limbs, + bq[l][src(i)], + out when accumulating).
// DN > 0: the digit count as a constant, so the 3 DN loads of a word are all
// issued before its products; DN = 0 takes dnum_rt.
template <int DN>
__global__ void k_ks_inner_b(const KsJobs J, int dnum_rt, int level, int L, int K, int logN,
                             const u64 *__restrict__ pmod, int accumulate, const PrimeInfo *__restrict__ pinfo)
{
    pdl_begin();
    const int dnum = DN > 0 ? DN : dnum_rt;
    const int jb = blockIdx.y;
    u64 *__restrict__ out = J.out[jb];
    const u64 *__restrict__ dig = J.dig[jb];
    const u64 *__restrict__ key = J.key[jb];
    const u64 *__restrict__ c0 = J.c0[jb];
    const u64 *__restrict__ bq = J.bq[jb];
    const u64 galois = J.gal[jb];
    const int kl = J.kl[jb];
    const size_t N = (size_t)1 << logN;
    const int nl = level + 1 + K, nK = kl + 1 + K;
    const size_t total = (size_t)nl * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx >> logN);
        const int i = (int)(idx & (N - 1));
        const int pid = l <= level ? l : L + 1 + (l - level - 1);
        const int kx = key_limb(pid, kl, L);
        const PrimeInfo pi = pinfo[pid];
        const int src = galois == 1 ? i : auto_src_b(i, logN, galois);
        Acc128 a0, a1;
#pragma unroll
        for (int j = 0; j < dnum; j++) {
            const u64 d = dig[((size_t)j * nl + l) * N + src];
            a0.mac(d, key[((size_t)(2 * j) * nK + kx) * N + i], pi.q);
            a1.mac(d, key[((size_t)(2 * j + 1) * nK + kx) * N + i], pi.q);
        }
        u64 r0 = a0.reduce(pi.q, pi.qinv);
        u64 r1 = a1.reduce(pi.q, pi.qinv);
        if (c0 && l <= level) r0 = add_mod(r0, mont_mul(c0[(size_t)l * N + src], pmod[pid], pi.q, pi.qinv), pi.q);
        if (bq) r0 = add_mod(r0, bq[(size_t)l * N + src], pi.q);
        if (accumulate) {
            r0 = add_mod(r0, out[idx], pi.q);
            r1 = add_mod(r1, out[total + idx], pi.q);
        }
        out[idx] = r0;
        out[total + idx] = r1;
    }
}

struct AutoJobs {
    int n;
    u64 *o[BJ];
    const u64 *a[BJ];
    u64 gal[BJ];
};

__global__ void k_auto_b(const AutoJobs J, int logN, size_t total)
{
    pdl_begin();
    u64 *__restrict__ o = J.o[blockIdx.y];
    const u64 *__restrict__ a = J.a[blockIdx.y];
    const u64 g = J.gal[blockIdx.y];
    const size_t N = (size_t)1 << logN;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t base = idx & ~(N - 1);
        o[idx] = a[base + auto_src_b((int)(idx & (N - 1)), logN, g)];
    }
}

// rescale helper of k_rescale_spread, one job per polynomial: the dropped
// limb (coefficient form) -> its centred remainder on limbs 0..level-1
struct SpreadJobs {
    int n;
    u64 *o[BJ];
    const u64 *last[BJ];
};
__global__ void k_spread_b(const SpreadJobs J, const u64 *__restrict__ tab, int nP, int logN, size_t total,
                           const PrimeInfo *__restrict__ pinfo)
{
    pdl_begin();
    u64 *__restrict__ out = J.o[blockIdx.y];
    const u64 *__restrict__ last = J.last[blockIdx.y];
    const size_t N = (size_t)1 << logN;
    const u64 ql = tab[2 * nP];
    const u64 half = (ql - 1) >> 1;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx >> logN);
        const u64 q = pinfo[l].q;
        const u64 x = last[idx & (N - 1)];
        const u64 xm = x < q ? x : x % q;
        out[idx] = x <= half ? xm : sub_mod(xm, tab[nP + l], q);
    }
}

// ------------------------------------------------------------ launch helpers
void ew_b(Ctx *c, int op, const std::vector<u64 *> &o, const std::vector<const u64 *> &a,
          const std::vector<const u64 *> &b, int n_limbs, LimbMap map)
{
    const size_t total = (size_t)n_limbs * c->N;
    if (!total || o.empty()) return;
    KTimer kt(c, "elementwise", 24.0 * total * o.size());
    for (size_t s = 0; s < o.size(); s += BJ) {
        EwJobs J;
        J.n = (int)std::min<size_t>(BJ, o.size() - s);
        for (int j = 0; j < J.n; j++) {
            J.o[j] = o[s + j];
            J.a[j] = a[s + j];
            J.b[j] = b[s + j];
        }
        launch(c, k_ew_b, dim3(gx_for(total, J.n), J.n), TPB, 0, J, c->logN, total, c->d_pinfo.as<PrimeInfo>(), map,
               op);
        c->launches++;
    }
    CUDA_CHECK(cudaGetLastError());
}

void copy_b(Ctx *c, const std::vector<u64 *> &o, const std::vector<const u64 *> &a, const std::vector<u64> &words)
{
    if (o.empty()) return;
    double bytes = 0;
    u64 mx = 0;
    for (u64 w : words) {
        bytes += 16.0 * w;
        mx = std::max(mx, w);
    }
    KTimer kt(c, "elementwise", bytes);
    for (size_t s = 0; s < o.size(); s += BJ) {
        CopyJobs J;
        J.n = (int)std::min<size_t>(BJ, o.size() - s);
        for (int j = 0; j < J.n; j++) {
            J.o[j] = o[s + j];
            J.a[j] = a[s + j];
            J.words[j] = words[s + j];
        }
        launch(c, k_copy_b, dim3(gx_for(mx, J.n), J.n), TPB, 0, J);
        c->launches++;
    }
    CUDA_CHECK(cudaGetLastError());
}

struct KsJob {
    u64 *out;
    const u64 *dig;
    const SwitchKey *key;
    u64 gal;
    const u64 *c0;
    const u64 *bq;
};

using KsInnerB = void (*)(const KsJobs, int, int, int, int, int, const u64 *, int, const PrimeInfo *);

KsInnerB ks_inner_kernel(int dnum)
{
    static const KsInnerB fns[] = {k_ks_inner_b<0>, k_ks_inner_b<1>, k_ks_inner_b<2>, k_ks_inner_b<3>,
                                   k_ks_inner_b<4>, k_ks_inner_b<5>, k_ks_inner_b<6>, k_ks_inner_b<7>,
                                   k_ks_inner_b<8>, k_ks_inner_b<9>};
    return dnum >= 1 && dnum <= 9 ? fns[dnum] : fns[0];
}

void ks_inner_b(Ctx *c, const std::vector<KsJob> &jobs, int level, bool accumulate)
{
    if (jobs.empty()) return;
    const int dnum = c->dnum(level);
    const size_t total = (size_t)(level + 1 + c->K) * c->N;
    double bytes = 0;
    for (auto &j : jobs)
        bytes += 8.0 * (total * (3.0 * dnum + (accumulate ? 4 : 2) + (j.bq ? 1 : 0)) +
                        (j.c0 ? (double)(level + 1) * c->N : 0.0));
    KTimer kt(c, "ks_inner_auto", bytes);
    for (size_t s = 0; s < jobs.size(); s += BJ) {
        KsJobs J;
        J.n = (int)std::min<size_t>(BJ, jobs.size() - s);
        for (int j = 0; j < J.n; j++) {
            const KsJob &x = jobs[s + j];
            J.out[j] = x.out;
            J.dig[j] = x.dig;
            HCHECK(x.key->level >= level, HELRM_E_NOKEY, "switching key generated below the level of its use");
            J.key[j] = x.key->data.u();
            J.kl[j] = x.key->level;
            J.c0[j] = x.c0;
            J.bq[j] = x.bq;
            J.gal[j] = x.gal;
        }
        launch(c, ks_inner_kernel(dnum), dim3(gx_for(total, J.n), J.n), TPB, 0, J, dnum, level, c->L, c->K, c->logN,
               c->d_pmod_mont.u(), accumulate ? 1 : 0, c->d_pinfo.as<PrimeInfo>());
        c->launches++;
    }
    CUDA_CHECK(cudaGetLastError());
}

void auto_b(Ctx *c, const std::vector<u64 *> &o, const std::vector<const u64 *> &a, const std::vector<u64> &gal,
            int n_limbs)
{
    const size_t total = (size_t)n_limbs * c->N;
    if (!total || o.empty()) return;
    KTimer kt(c, "automorphism", 16.0 * total * o.size());
    for (size_t s = 0; s < o.size(); s += BJ) {
        AutoJobs J;
        J.n = (int)std::min<size_t>(BJ, o.size() - s);
        for (int j = 0; j < J.n; j++) {
            J.o[j] = o[s + j];
            J.a[j] = a[s + j];
            J.gal[j] = gal[s + j];
        }
        launch(c, k_auto_b, dim3(gx_for(total, J.n), J.n), TPB, 0, J, c->logN, total);
        c->launches++;
    }
    CUDA_CHECK(cudaGetLastError());
}

// ------------------------------------------------------------ batched CKKS steps
using CtVec = std::vector<Ciphertext *>;
using CCtVec = std::vector<const Ciphertext *>;

struct Owned {   // owns the ciphertexts of one batched value
    std::vector<std::unique_ptr<Ciphertext>> v;
    CCtVec craw() const
    {
        CCtVec r;
        for (auto &p : v) r.push_back(p.get());
        return r;
    }
};

// ModUp (iNTT, fast base conversion of every digit, NTT of the converted
// limbs) of several polynomials at `level`, as ks_modup.
void modup_b(Ctx *c, const std::vector<const u64 *> &polys, int level, const std::vector<u64 *> &digits)
{
    const int N = c->N, nq = level + 1, nl = nq + c->K, dnum = c->dnum(level);
    const size_t B = polys.size();
    DevMem coef(c, B * nq * N * 8);
    std::vector<k::NttLimb> inv, fwd;   // the base conversion runs inside the two transforms
    for (size_t q = 0; q < B; q++) modup_limbs(c, level, polys[q], coef.u() + q * nq * N, digits[q], inv, fwd);
    k::ntt_run(c, inv, true, nullptr);
    std::vector<u64 *> co;
    std::vector<const u64 *> ca;
    std::vector<u64> cw;
    for (size_t q = 0; q < B; q++)
        for (int j = 0; j < dnum; j++) {   // each digit keeps its own limbs as they are
            const int lo = c->digit_lo(j), hi = c->digit_hi(j, level);
            co.push_back(digits[q] + ((size_t)j * nl + lo) * N);
            ca.push_back(polys[q] + (size_t)lo * N);
            cw.push_back((u64)(hi - lo) * N);
        }
    copy_b(c, co, ca, cw);
    k::ntt_run(c, fwd, false, nullptr);
}

// ModDown of `halves` QP polynomials per entry (u[q] = [halves][nl][N]), as
// ks_moddown2 / ks_moddown: out_h = (u_h - FBC_{P->Q}([u_h]_P)) P^-1 (+ add_h).
void moddown_b(Ctx *c, const std::vector<const u64 *> &u, int level, int halves, const std::vector<u64 *> &out0,
               const std::vector<u64 *> &out1, const std::vector<const u64 *> &add0,
               const std::vector<const u64 *> &add1)
{
    const int N = c->N, nq = level + 1, K = c->K, nl = nq + K;
    const size_t B = u.size();
    DevMem pc(c, B * halves * K * N * 8), y(c, B * halves * nq * N * 8);
    std::vector<k::NttLimb> inv, fwd;   // the base conversion runs inside the two transforms
    for (size_t q = 0; q < B; q++)
        for (int h = 0; h < halves; h++)
            moddown_limbs(c, level, u[q] + (size_t)h * nl * N, pc.u() + (q * halves + h) * K * N,
                          y.u() + (q * halves + h) * nq * N, h ? out1[q] : out0[q], h ? add1[q] : add0[q], inv, fwd);
    k::ntt_run(c, inv, true, nullptr);
    k::ntt_run(c, fwd, false, c->d_pinv_mont.u());
}

// A ModDown of both halves followed by a rescale, merged into one pair of
// transforms: out = rescale((u - FBC([u]_P)) P^-1 + add) at level - 1 with
// scale / q_level (NttRescale: the same residues as moddown_b + rescale_b).
// u[q] = [2][level+1+K][N]; add0/add1 entries may be null.
Owned moddown_rescale_b(Ctx *c, const std::vector<const u64 *> &u, int level, const std::vector<double> &scale,
                        const std::vector<const u64 *> &add0, const std::vector<const u64 *> &add1)
{
    HCHECK(level >= 1, HELRM_E_LEVEL, "no level left to rescale");
    const int N = c->N, nq = level + 1, K = c->K, nl = nq + K;
    const size_t B = u.size();
    const BConvTable &t = c->moddown_table(level);
    const LimbMap m = c->qmap(level);
    Owned o;
    for (size_t q = 0; q < B; q++) o.v.emplace_back(new_ct(c, level - 1, scale[q] / (double)c->primes[level]));
    // per half: K P-limbs (scaled for the conversion), the top Q-limb of u and of the addend (plain)
    DevMem pc(c, B * 2 * K * N * 8), top(c, B * 2 * 2 * N * 8), y(c, B * 2 * level * N * 8);
    std::vector<k::NttLimb> inv, fwd;
    for (size_t q = 0; q < B; q++)
        for (int h = 0; h < 2; h++) {
            const size_t qh = q * 2 + h;
            const u64 *uh = u[q] + (size_t)h * nl * N;
            const u64 *ad = h ? add1[q] : add0[q];
            u64 *pch = pc.u() + qh * K * N;
            for (int i = 0; i < K; i++) {
                k::NttLimb x{uh + (size_t)(nq + i) * N, pch + (size_t)i * N, m.pid(nq + i), nullptr, nullptr, nullptr};
                x.scal = t.scale(i);
                inv.push_back(x);
            }
            u64 *ut = top.u() + (qh * 2) * N, *at = top.u() + (qh * 2 + 1) * N;
            inv.push_back({uh + (size_t)level * N, ut, level, nullptr, nullptr, nullptr});
            if (ad) inv.push_back({ad + (size_t)level * N, at, level, nullptr, nullptr, nullptr});
            u64 *oh = h ? o.v[q]->c1() : o.v[q]->c0();
            for (int i = 0; i < level; i++) {
                k::NttLimb x{pch, y.u() + (qh * level + i) * N, i, uh + (size_t)i * N, oh + (size_t)i * N,
                             ad ? ad + (size_t)i * N : nullptr};
                x.fbc_n = K;
                x.fbc_h = t.hcol(i);
                x.fbc_hs = t.n_dst;
                x.rs_u = ut;
                x.rs_add = ad ? at : nullptr;
                fwd.push_back(x);
            }
        }
    k::ntt_run(c, inv, true, nullptr);
    k::NttRescale rs;
    rs.hl = t.hcol(level);
    rs.hls = t.n_dst;
    rs.lp = level;
    rs.pmod = c->d_pmod_mont.u();
    rs.qlmod = c->rescale_table(level) + c->nP();
    rs.pinv = c->d_pinv_mont.u();
    rs.ep_scal = c->moddown_rescale_table(level);
    rs.add_off = c->nP();
    k::ntt_run_rescale(c, fwd, rs);
    return o;
}

// rescale of every ciphertext (all at the same level), as ct_rescale
Owned rescale_b(Ctx *c, const CCtVec &a)
{
    Owned o;
    if (a.empty()) return o;
    const int l = a[0]->level, N = c->N;
    const size_t B = a.size();
    HCHECK(l >= 1, HELRM_E_LEVEL, "no level left to rescale");
    for (auto *x : a) {
        HCHECK(x->level == l, HELRM_E_LEVEL, "batched rescale needs one level");
        o.v.emplace_back(new_ct(c, l - 1, x->scale / (double)c->primes[l]));
    }
    DevMem last(c, B * 2 * N * 8), r(c, B * 2 * l * N * 8);
    std::vector<k::NttLimb> v;
    for (size_t q = 0; q < B; q++)
        for (int h = 0; h < 2; h++)
            v.push_back({(h ? a[q]->c1() : a[q]->c0()) + (size_t)l * N, last.u() + (q * 2 + h) * N, l, nullptr,
                         nullptr, nullptr});
    k::ntt_run(c, v, true, nullptr);
    const size_t total = (size_t)l * N;
    {
        KTimer kt(c, "rescale_spread", 8.0 * 2 * B * (total + N));
        for (size_t s = 0; s < 2 * B; s += BJ) {
            SpreadJobs J;
            J.n = (int)std::min<size_t>(BJ, 2 * B - s);
            for (int j = 0; j < J.n; j++) {
                J.o[j] = r.u() + (s + j) * l * N;
                J.last[j] = last.u() + (s + j) * N;
            }
            launch(c, k_spread_b, dim3(gx_for(total, J.n), J.n), TPB, 0, J, c->rescale_table(l), c->nP(), c->logN,
                   total, c->d_pinfo.as<PrimeInfo>());
            c->launches++;
        }
        CUDA_CHECK(cudaGetLastError());
    }
    v.clear();
    for (size_t q = 0; q < B; q++)
        for (int h = 0; h < 2; h++)
            for (int i = 0; i < l; i++) {
                u64 *ri = r.u() + ((q * 2 + h) * l + i) * N;
                v.push_back({ri, ri, i, (h ? a[q]->c1() : a[q]->c0()) + (size_t)i * N,
                             (h ? o.v[q]->c1() : o.v[q]->c0()) + (size_t)i * N, nullptr});
            }
    k::ntt_run(c, v, false, c->rescale_table(l));
    return o;
}

Owned add_b(Ctx *c, const CCtVec &a, const CCtVec &b)
{
    Owned o;
    std::vector<u64 *> oo;
    std::vector<const u64 *> aa, bb;
    for (size_t q = 0; q < a.size(); q++) {
        HCHECK(a[q]->level == b[q]->level && a[q]->level == a[0]->level, HELRM_E_LEVEL, "ciphertext levels differ");
        HCHECK(std::fabs(a[q]->scale - b[q]->scale) <= 1e-9 * a[q]->scale, HELRM_E_SCALE, "ciphertext scales differ");
        o.v.emplace_back(new_ct(c, a[q]->level, a[q]->scale));
        oo.push_back(o.v[q]->data.u());
        aa.push_back(a[q]->data.u());
        bb.push_back(b[q]->data.u());
    }
    if (a.empty()) return o;
    const int l = a[0]->level;
    ew_b(c, B_ADD, oo, aa, bb, 2 * (l + 1), c->qmap(l, 0, l + 1));
    return o;
}

Owned add_pt_b(Ctx *c, const CCtVec &a, const Plaintext *pt)
{
    HCHECK(pt->form == PT_PLAIN, HELRM_E_INVAL, "plaintext is in multiplier form");
    Owned o;
    if (a.empty()) return o;
    const int l = a[0]->level, nq = l + 1;
    HCHECK(pt->level >= l, HELRM_E_LEVEL, "plaintext level below ciphertext level");
    std::vector<u64 *> oo, co;
    std::vector<const u64 *> aa, bb, ca;
    std::vector<u64> cw;
    for (size_t q = 0; q < a.size(); q++) {
        HCHECK(a[q]->level == l, HELRM_E_LEVEL, "batched op needs one level");
        HCHECK(std::fabs(a[q]->scale - pt->scale) <= 1e-9 * a[q]->scale, HELRM_E_SCALE, "plaintext scale differs");
        o.v.emplace_back(new_ct(c, l, a[q]->scale));
        oo.push_back(o.v[q]->c0());
        aa.push_back(a[q]->c0());
        bb.push_back(pt->data.u());
        co.push_back(o.v[q]->c1());
        ca.push_back(a[q]->c1());
        cw.push_back((u64)nq * c->N);
    }
    ew_b(c, B_ADD, oo, aa, bb, nq, c->qmap(l));
    copy_b(c, co, ca, cw);
    return o;
}

// products of every ciphertext a[q] with every plaintext pts[i]: out[q * n_pt + i]
Owned mul_pt_b(Ctx *c, const CCtVec &a, const std::vector<const Plaintext *> &pts)
{
    Owned o;
    if (a.empty() || pts.empty()) return o;
    const int l = a[0]->level, nq = l + 1;
    const int form = pts[0]->form;
    std::vector<u64 *> oo;
    std::vector<const u64 *> aa, bb;
    for (size_t q = 0; q < a.size(); q++) {
        HCHECK(a[q]->level == l, HELRM_E_LEVEL, "batched op needs one level");
        for (const Plaintext *pt : pts) {
            HCHECK(pt->level >= l && !pt->qp && pt->form == form, HELRM_E_LEVEL, "plaintext level below ciphertext level");
            std::unique_ptr<Ciphertext> x(new_ct(c, l, a[q]->scale * pt->scale));
            for (int h = 0; h < 2; h++) {
                oo.push_back(h ? x->c1() : x->c0());
                aa.push_back(h ? a[q]->c1() : a[q]->c0());
                bb.push_back(pt->data.u());
            }
            o.v.push_back(std::move(x));
        }
    }
    ew_b(c, form == PT_MONT ? B_MULM : B_MULP, oo, aa, bb, nq, c->qmap(l));
    return o;
}

// rotations of every a[q] by every step (one ModUp per query, shared by its
// steps): out[q * S + s], as ct_rotate_hoisted
// X -> X^g for every Galois element of gals on every query's ciphertext,
// sharing one ModUp per query (hoisted), as ct_rotate_hoisted / ct_apply_galois
Owned galois_b(Ctx *c, const std::vector<const EvalKey *> &evk, const CCtVec &a, const std::vector<u64> &gals)
{
    Owned o;
    if (a.empty()) return o;
    const int l = a[0]->level, N = c->N, nq = l + 1, nl = nq + c->K, dnum = c->dnum(l);
    const size_t B = a.size(), S = gals.size();
    const size_t dplane = (size_t)dnum * nl * N, uplane = (size_t)2 * nl * N;
    for (auto *x : a) HCHECK(x->level == l, HELRM_E_LEVEL, "batched rotation needs one level");
    std::vector<const SwitchKey *> keys(B * S, nullptr);
    for (size_t q = 0; q < B; q++)
        for (size_t s = 0; s < S; s++)
            if (gals[s] != 1) keys[q * S + s] = rot_key(evk[q], gals[s], l);
    DevMem digits(c, B * dplane * 8), u(c, B * S * uplane * 8);
    std::vector<const u64 *> c1s;
    std::vector<u64 *> dg;
    for (size_t q = 0; q < B; q++) {
        c1s.push_back(a[q]->c1());
        dg.push_back(digits.u() + q * dplane);
    }
    modup_b(c, c1s, l, dg);
    std::vector<KsJob> jobs;
    std::vector<u64 *> ao, co;
    std::vector<const u64 *> aa, ca, uu, add0;
    std::vector<u64> ag, cw;
    std::vector<u64 *> o0, o1;
    for (size_t q = 0; q < B; q++)
        for (size_t s = 0; s < S; s++) {
            const u64 g = gals[s];
            std::unique_ptr<Ciphertext> x(new_ct(c, l, a[q]->scale));
            if (g == 1) {
                co.push_back(x->data.u());
                ca.push_back(a[q]->data.u());
                cw.push_back((u64)2 * nq * N);
            } else {
                u64 *uq = u.u() + (q * S + s) * uplane;
                jobs.push_back({uq, dg[q], keys[q * S + s], g, nullptr, nullptr});
                ao.push_back(x->c0());
                aa.push_back(a[q]->c0());
                ag.push_back(g);
                uu.push_back(uq);
                o0.push_back(x->c0());
                o1.push_back(x->c1());
                add0.push_back(x->c0());
            }
            o.v.push_back(std::move(x));
        }
    copy_b(c, co, ca, cw);
    ks_inner_b(c, jobs, l, false);
    auto_b(c, ao, aa, ag, nq);
    moddown_b(c, uu, l, 2, o0, o1, add0, std::vector<const u64 *>(uu.size(), nullptr));   // phi(c0) + ModDown(u)
    return o;
}

Owned rotate_b(Ctx *c, const std::vector<const EvalKey *> &evk, const CCtVec &a, const std::vector<int> &steps)
{
    std::vector<u64> gals;
    for (int st : steps) gals.push_back(c->galois(st));
    return galois_b(c, evk, a, gals);
}

// relinearisation of (d0, d1, d2) per query, as ct_relin; with rescale, the
// result is also rescaled (the ModDown and the rescale merged)
Owned relin_b(Ctx *c, const std::vector<const EvalKey *> &evk, const std::vector<const u64 *> &d012, int level,
              double scale, bool rescale = false)
{
    Owned o;
    const int N = c->N, nq = level + 1, nl = nq + c->K, dnum = c->dnum(level);
    const size_t B = d012.size(), plane = (size_t)nq * N, dplane = (size_t)dnum * nl * N, uplane = (size_t)2 * nl * N;
    for (auto *e : evk) relin_key(e, level);
    DevMem digits(c, B * dplane * 8), u(c, B * uplane * 8);
    std::vector<const u64 *> d2, uu, a0, a1;
    std::vector<u64 *> dg, o0, o1;
    for (size_t q = 0; q < B; q++) {
        d2.push_back(d012[q] + 2 * plane);
        dg.push_back(digits.u() + q * dplane);
    }
    modup_b(c, d2, level, dg);
    std::vector<KsJob> jobs;
    for (size_t q = 0; q < B; q++) {
        u64 *uq = u.u() + q * uplane;
        jobs.push_back({uq, dg[q], relin_key(evk[q], level), 1, nullptr, nullptr});
        uu.push_back(uq);
        a0.push_back(d012[q]);
        a1.push_back(d012[q] + plane);
    }
    ks_inner_b(c, jobs, level, false);
    if (rescale) return moddown_rescale_b(c, uu, level, std::vector<double>(B, scale), a0, a1);
    for (size_t q = 0; q < B; q++) {
        o.v.emplace_back(new_ct(c, level, scale));
        o0.push_back(o.v[q]->c0());
        o1.push_back(o.v[q]->c1());
    }
    moddown_b(c, uu, level, 2, o0, o1, a0, a1);   // (d0, d1) + ModDown(u)
    return o;
}

void tensor_b(Ctx *c, const std::vector<u64 *> &d, const CCtVec &a, const CCtVec &b, bool accumulate)
{
    if (a.empty()) return;
    const int l = a[0]->level;
    const size_t total = (size_t)(l + 1) * c->N;
    KTimer kt(c, "tensor", (accumulate ? 10.0 : 7.0) * 8 * total * a.size());
    for (size_t s = 0; s < a.size(); s += BJ) {
        TensorJobs J;
        J.n = (int)std::min<size_t>(BJ, a.size() - s);
        for (int j = 0; j < J.n; j++) {
            HCHECK(a[s + j]->level == l && b[s + j]->level == l, HELRM_E_LEVEL, "ciphertext levels differ");
            J.d[j] = d[s + j];
            J.a0[j] = a[s + j]->c0();
            J.a1[j] = a[s + j]->c1();
            J.b0[j] = b[s + j]->c0();
            J.b1[j] = b[s + j]->c1();
        }
        launch(c, k_tensor_b, dim3(gx_for(total, J.n), J.n), TPB, 0, J, c->logN, total, c->d_pinfo.as<PrimeInfo>(),
               c->qmap(l), accumulate ? 1 : 0);
        c->launches++;
    }
    CUDA_CHECK(cudaGetLastError());
}

// a * a, relinearised and rescaled (the x^2 activation), as ct_mul(a, a)
Owned square_b(Ctx *c, const std::vector<const EvalKey *> &evk, const CCtVec &a)
{
    const int l = a[0]->level;
    HCHECK(l >= 1, HELRM_E_LEVEL, "no level left for a multiplication");
    const size_t B = a.size(), per = (size_t)3 * (l + 1) * c->N;
    DevMem d(c, B * per * 8);
    std::vector<u64 *> dd;
    std::vector<const u64 *> cd;
    for (size_t q = 0; q < B; q++) {
        dd.push_back(d.u() + q * per);
        cd.push_back(d.u() + q * per);
    }
    tensor_b(c, dd, a, a, false);
    return relin_b(c, evk, cd, l, a[0]->scale * a[0]->scale, true);
}

// every ciphertext taken down to `level` (the first level + 1 limbs of each half)
Owned drop_b(Ctx *c, const CCtVec &a, int level)
{
    Owned o;
    std::vector<u64 *> out;
    std::vector<const u64 *> in;
    std::vector<u64> words;
    for (auto *x : a) {
        HCHECK(level >= 0 && level <= x->level, HELRM_E_LEVEL, "cannot raise the level");
        o.v.emplace_back(new_ct(c, level, x->scale));
        for (int h = 0; h < 2; h++) {
            out.push_back(h ? o.v.back()->c1() : o.v.back()->c0());
            in.push_back(h ? x->c1() : x->c0());
            words.push_back((u64)(level + 1) * c->N);
        }
    }
    copy_b(c, out, in, words);
    return o;
}

}  // namespace

// The polynomial of `plan` on every query's ciphertext (poly.cu gives the
// schedule): the needed powers by merged ct x ct products, each term times its
// integer constant at the common level, the sum, one rescale, then a_0.
std::vector<Ciphertext *> poly_b(Ctx *c, const std::vector<const EvalKey *> &evk, const CCtVec &x,
                                 const ActPlan &plan)
{
    const size_t B = x.size();
    HCHECK(B >= 1 && evk.size() == B, HELRM_E_INVAL, "one key set per ciphertext");
    for (auto *ct : x)
        HCHECK(ct->level == plan.in_level && ct->scale == plan.in_scale, HELRM_E_SCALE,
               "ciphertext level or scale differs from the polynomial plan's");
    std::map<int, Owned> own;
    std::map<int, CCtVec> pw;
    pw[1] = x;
    auto at_level = [&](const CCtVec &v, int l, Owned &keep) -> CCtVec {
        if (v[0]->level == l) return v;
        keep = drop_b(c, v, l);
        return keep.craw();
    };
    for (const auto &t : plan.tree) {
        const int lvl = std::min(pw[t[1]][0]->level, pw[t[2]][0]->level);
        Owned ka, kb;
        const CCtVec A = at_level(pw[t[1]], lvl, ka), Bv = at_level(pw[t[2]], lvl, kb);
        const size_t per = (size_t)3 * (lvl + 1) * c->N;
        DevMem d(c, B * per * 8);
        std::vector<u64 *> dd;
        std::vector<const u64 *> cd;
        for (size_t q = 0; q < B; q++) {
            dd.push_back(d.u() + q * per);
            cd.push_back(d.u() + q * per);
        }
        tensor_b(c, dd, A, Bv, false);
        own[t[0]] = relin_b(c, evk, cd, lvl, A[0]->scale * Bv[0]->scale, true);
        pw[t[0]] = own[t[0]].craw();
    }
    const int lc = plan.level_c;
    Owned acc;
    for (const auto &term : plan.terms) {
        Owned keep;
        const CCtVec v = at_level(pw[term.k], lc, keep);
        Owned m;
        for (size_t q = 0; q < B; q++) {
            m.v.emplace_back(new_ct(c, lc, term.scale));
            k::mul_scalar_mont(c, m.v[q]->data.u(), v[q]->data.u(), term.mont.u(), 2 * (lc + 1),
                               c->qmap(lc, 0, lc + 1));
        }
        acc = acc.v.empty() ? std::move(m) : add_b(c, acc.craw(), m.craw());
    }
    Owned y = rescale_b(c, acc.craw());
    if (plan.a0.ptr)
        for (auto &ct : y.v) k::add_scalar(c, ct->c0(), ct->c0(), plan.a0.u(), ct->level + 1, c->qmap(ct->level));
    std::vector<Ciphertext *> out;
    for (auto &p : y.v) out.push_back(p.release());
    return out;
}

// ------------------------------------------------------------------ the batch
struct Batch : Handle {
    Ctx *ctx;
    const Model *model;
    std::vector<const EvalKey *> evk;
    std::map<const PtMatrix *, DevMem> keytab;   // [B][64] baby-step key pointers, then [B][64] their levels
    // graph replay: the whole server path captured once on fixed buffers
    bool use_graph = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t gstream = nullptr;            // the graph's own stream (a legacy default stream cannot be captured)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<std::unique_ptr<Ciphertext>> g_dense, g_sel, g_out;
    Batch(Ctx *c) : Handle(KIND_BATCH), ctx(c) {}
    ~Batch() override
    {
        if (gstream) cudaStreamSynchronize(gstream);
        if (exec) cudaGraphExecDestroy(exec);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (gstream) cudaStreamDestroy(gstream);
    }
};

static void batch_keytab(Batch *bt, const PtMatrix *m)
{
    Ctx *c = bt->ctx;
    if (!(m->n1 <= 64 && m->n2 <= 8)) return;
    std::vector<char> need(m->n1, 0);
    for (auto &gb : m->gb) need[gb.second] = 1;
    const size_t B = bt->evk.size();
    std::vector<const u64 *> tab(B * 64, nullptr);
    std::vector<int> lv(B * 64, 0);
    for (size_t q = 0; q < B; q++)
        for (int b = 1; b < m->n1; b++)
            if (need[b]) {
                const SwitchKey *k = rot_key(bt->evk[q], c->galois(b), m->level);
                tab[q * 64 + b] = k->data.u();
                lv[q * 64 + b] = k->level;
            }
    const size_t pb = tab.size() * sizeof(u64 *);
    DevMem d(c, pb + lv.size() * sizeof(int));
    CUDA_CHECK(cudaMemcpyAsync(d.ptr, tab.data(), pb, cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaMemcpyAsync((char *)d.ptr + pb, lv.data(), lv.size() * sizeof(int), cudaMemcpyHostToDevice,
                               c->stream));
    bt->keytab[m] = std::move(d);
}

Batch *batch_create(Ctx *c, const Model *m, const std::vector<const EvalKey *> &evk)
{
    HCHECK(!evk.empty(), HELRM_E_INVAL, "empty batch");
    std::unique_ptr<Batch> b(new Batch(c));
    b->model = m;
    b->evk = evk;
    for (auto &L : m->bottom) batch_keytab(b.get(), L.pm.get());
    for (PtMatrix *pm : m->emb_mats()) batch_keytab(b.get(), pm);
    for (auto &L : m->top) batch_keytab(b.get(), L.pm.get());
    for (const Model::BootPoint *bp : m->boot_points())
        for (PtMatrix *pm : bp->b->matrices()) batch_keytab(b.get(), pm);
    // (the host tables were staged by the copies themselves: nothing to wait for)
    return b.release();
}

// y = W x for every query (double-hoisted BSGS, rescale, folds), as matvec
// The baby-step half of the batch's products by matrix m (the fused kernel's
// shapes): one ModUp per query, then the hoisted baby steps and the BSGS MAC
// into inner[q][g][2][plane]; need_g[g] is set for the giant steps with
// diagonals.
static void baby_products_b(Ctx *c, const Batch *bt, const PtMatrix *m, const CCtVec &in, u64 *inner,
                            std::vector<char> &need_g)
{
    const size_t B = in.size();
    const int l = in[0]->level, N = c->N, nl = l + 1 + c->K, dnum = c->dnum(l);
    auto kt = bt->keytab.find(m);
    const size_t plane = (size_t)nl * N, dplane = (size_t)dnum * plane;
    std::vector<char> need_b(m->n1, 0);
    need_g.assign(m->n2, 0);
    for (auto &gb : m->gb) {
        need_b[gb.second] = 1;
        need_g[gb.first] = 1;
    }
    bool any_baby = false;
    int n_keys = 0;
    for (int b = 1; b < m->n1; b++) {
        any_baby |= need_b[b] != 0;
        n_keys += need_b[b] ? 1 : 0;
    }
    DevMem digits(c, B * dplane * 8);
    std::vector<u64 *> dg;
    std::vector<const u64 *> c1s;
    for (size_t q = 0; q < B; q++) {
        dg.push_back(digits.u() + q * dplane);
        c1s.push_back(in[q]->c1());
    }
    if (any_baby) modup_b(c, c1s, l, dg);
    const size_t iq = (size_t)m->n2 * 2 * plane;   // inner products of one query
    std::vector<u64> gals(m->n1, 1);
    for (int b = 1; b < m->n1; b++)
        if (need_b[b]) gals[b] = c->galois(b);
    std::vector<k::BsgsQuery> qs;
    for (size_t q = 0; q < B; q++) qs.push_back({inner + q * iq, dg[q], in[q]->c0(), in[q]->c1()});
    k::bsgs_tma_batch(c, qs, kt->second.as<const u64 *const>(),
                      (const int *)((const char *)kt->second.ptr + B * 64 * sizeof(u64 *)), gals.data(),
                      m->d_ptrs.as<const u64 *const>(),
                      m->d_gb_index.as<int>(), (int)m->gb.size(), n_keys, m->n1, m->n2, l);
}

// sum_k W_k x_k for every query of the batch, the matrices of one shape
// (reading R31: the baby-step products are added over QP and the sum takes
// one set of giant steps, one ModDown + rescale and one set of folds); with
// one matrix, the batch's product by it.  in[k] holds the B ciphertexts
// multiplied by ms[k].
static Owned matvec_sum_b(Ctx *c, const Batch *bt, const std::vector<const PtMatrix *> &ms,
                          const std::vector<CCtVec> &in)
{
    const PtMatrix *m = ms[0];
    const size_t B = in[0].size();
    const int l = in[0][0]->level, N = c->N, nq = l + 1, nl = nq + c->K, dnum = c->dnum(l);
    for (size_t k2 = 0; k2 < ms.size(); k2++) {
        HCHECK(same_shape(ms[k2], m) && in[k2].size() == B, HELRM_E_PARAM, "batched product sum: shapes differ");
        for (size_t q = 0; q < B; q++)
            HCHECK(in[k2][q]->level == m->level && in[k2][q]->scale == in[0][q]->scale, HELRM_E_LEVEL,
                   "ciphertext level or scale does not match the prepared matrix");
    }
    bool fused = true;
    for (auto *mk : ms) fused &= bt->keytab.count(mk) != 0;
    if (!fused) {   // shapes outside the fused kernel: the one-query path, query by query
        Owned o;
        for (size_t q = 0; q < B; q++) {
            std::vector<const Ciphertext *> xs;
            for (auto &v : in) xs.push_back(v[q]);
            o.v.emplace_back(matvec_sum(c, bt->evk[q], ms, xs));
        }
        return o;
    }
    const size_t plane = (size_t)nl * N, dplane = (size_t)dnum * plane;
    const size_t iq = (size_t)m->n2 * 2 * plane;   // inner products of one query
    DevMem inner(c, B * iq * 8);
    std::vector<char> need_g;
    if (ms.size() == 1) {
        baby_products_b(c, bt, m, in[0], inner.u(), need_g);
    } else {
        DevMem part(c, B * iq * 8);
        k::zero(c, inner.u(), B * iq);
        need_g.assign(m->n2, 0);
        std::vector<char> ng;
        for (size_t k2 = 0; k2 < ms.size(); k2++) {
            k::zero(c, part.u(), B * iq);
            baby_products_b(c, bt, ms[k2], in[k2], part.u(), ng);
            for (int g = 0; g < m->n2; g++) need_g[g] |= ng[g];
            k::add(c, inner.u(), inner.u(), part.u(), (int)(B * m->n2 * 2 * nl), c->qmap(l, 0, nl));
        }
    }
    std::vector<const SwitchKey *> gkey(B * m->n2, nullptr);
    for (size_t q = 0; q < B; q++)
        for (int g = 1; g < m->n2; g++)
            if (need_g[g]) gkey[q * m->n2 + g] = rot_key(bt->evk[q], c->galois(g * m->n1), l);
    // giant steps: ModDown the a-part of every (query, g > 0), ModUp them all,
    // then one key product per g adds phi(inner_g) into inner_0 of each query
    std::vector<int> gs;
    for (int g = 1; g < m->n2; g++)
        if (need_g[g]) gs.push_back(g);
    if (!need_g[0])
        for (size_t q = 0; q < B; q++) k::zero(c, inner.u() + q * iq, 2 * plane);
    if (!gs.empty()) {
        const size_t G = gs.size();
        DevMem c1q(c, B * G * (size_t)nq * N * 8), gdig(c, B * G * dplane * 8);
        std::vector<const u64 *> ua, c1v;
        std::vector<u64 *> o0, gd;
        for (size_t q = 0; q < B; q++)
            for (size_t t = 0; t < G; t++) {
                ua.push_back(inner.u() + q * iq + (size_t)gs[t] * 2 * plane + plane);
                o0.push_back(c1q.u() + (q * G + t) * nq * N);
                c1v.push_back(o0.back());
                gd.push_back(gdig.u() + (q * G + t) * dplane);
            }
        std::vector<const u64 *> none(ua.size(), nullptr);
        moddown_b(c, ua, l, 1, o0, o0, none, none);
        modup_b(c, c1v, l, gd);
        for (size_t t = 0; t < G; t++) {
            std::vector<KsJob> jobs;
            const u64 gal = c->galois(gs[t] * m->n1);
            for (size_t q = 0; q < B; q++)
                jobs.push_back({inner.u() + q * iq, gd[q * G + t], gkey[q * m->n2 + gs[t]], gal, nullptr,
                                inner.u() + q * iq + (size_t)gs[t] * 2 * plane});
            ks_inner_b(c, jobs, l, true);
        }
    }
    std::vector<const u64 *> acc, none(B, nullptr);
    std::vector<double> sc;
    for (size_t q = 0; q < B; q++) {
        acc.push_back(inner.u() + q * iq);
        sc.push_back(in[0][q]->scale * m->pt_scale);
    }
    Owned y = moddown_rescale_b(c, acc, l, sc, none, none);   // the final ModDown and the rescale, merged
    for (auto &p : y.v) p->scale = m->out_scale;
    for (auto &f : m->folds) {   // one level: the radix - 1 rotations hoisted, then added
        std::vector<int> steps;
        for (int d = 1; d < f.second; d++) steps.push_back(d * f.first);
        Owned r = rotate_b(c, bt->evk, y.craw(), steps);   // [q][step]
        for (size_t s = 0; s < steps.size(); s++) {
            CCtVec rs;
            for (size_t q = 0; q < B; q++) rs.push_back(r.v[q * steps.size() + s].get());
            y = add_b(c, y.craw(), rs);
        }
    }
    return y;
}

static Owned matvec_b(Ctx *c, const Batch *bt, const PtMatrix *m, const CCtVec &in)
{
    return matvec_sum_b(c, bt, {m}, {in});
}

static Owned dense_layer_b(Ctx *c, const Batch *bt, const Layer &L, const CCtVec &x)
{
    Owned y = matvec_b(c, bt, L.pm.get(), x);
    y = add_pt_b(c, y.craw(), L.bias.get());
    if (L.square && !L.act) y = square_b(c, bt->evk, y.craw());
    if (L.square && L.act) {   // the polynomial without a_0, then a_0 on the real outputs
        Owned p;
        for (auto *ct : poly_b(c, bt->evk, y.craw(), *L.act)) p.v.emplace_back(ct);
        y = L.act_const ? add_pt_b(c, p.craw(), L.act_const.get()) : std::move(p);
    }
    return y;
}

static Owned dot_interaction_b(Ctx *c, const Batch *bt, const Model *m, const CCtVec &z)
{
    const size_t B = z.size();
    const int S = m->S;
    std::vector<const Plaintext *> masks;
    for (auto &p : m->masks) masks.push_back(p.get());
    Owned zm = mul_pt_b(c, z, masks);                 // [q][i], i = 0..S
    Owned zr = rescale_b(c, zm.craw());
    for (auto &p : zr.v) p->scale = c->delta;
    CCtVec z1, A;                                      // A[q * S + s - 1] = z_q masked by mask s
    for (size_t q = 0; q < B; q++) {
        z1.push_back(zr.v[q * (S + 1)].get());
        for (int s = 1; s <= S; s++) A.push_back(zr.v[q * (S + 1) + s].get());
    }
    Owned r = rotate_b(c, bt->evk, z1, {-DIM * m->Bp});
    Owned zz = add_b(c, z1, r.craw());
    std::vector<int> steps;
    for (int s = 1; s <= S; s++) steps.push_back(DIM * s);
    Owned R = rotate_b(c, bt->evk, zz.craw(), steps);   // [q][s - 1]
    const int lvl = z1[0]->level;
    const size_t per = (size_t)3 * (lvl + 1) * c->N;
    DevMem d(c, B * per * 8);
    std::vector<u64 *> dd;
    std::vector<const u64 *> cd;
    for (size_t q = 0; q < B; q++) {
        dd.push_back(d.u() + q * per);
        cd.push_back(d.u() + q * per);
    }
    for (int s = 1; s <= S; s++) {
        CCtVec as, rs;
        for (size_t q = 0; q < B; q++) {
            as.push_back(A[q * S + s - 1]);
            rs.push_back(R.v[q * S + s - 1].get());
        }
        tensor_b(c, dd, as, rs, s > 1);
    }
    return relin_b(c, bt->evk, cd, lvl, c->delta * c->delta, true);
}

// a + v on every slot of every query's ciphertext (v as residues per prime id)
static Owned add_int_b(Ctx *c, const CCtVec &a, const DevMem &t)
{
    Owned o;
    for (auto *x : a) {
        o.v.emplace_back(new_ct(c, x->level, x->scale));
        k::add_scalar(c, o.v.back()->c0(), x->c0(), t.u(), x->level + 1, c->qmap(x->level));
        k::copy(c, o.v.back()->c1(), x->c1(), (size_t)(x->level + 1) * c->N);
    }
    return o;
}

// The bootstrap of boot.cu on every query's ciphertext, step by step for the
// whole batch (the same operations: ModRaise per query, then SubSum,
// CoeffToSlot and its conjugate, EvalMod and SlotToCoeff with the batched
// rotations, products and matvecs, whose CTAs of all queries that work on the
// same tile run together, so shared rows are read once); then dropped to the
// first level of the next segment.
static Owned boot_all(Ctx *c, const Batch *bt, const Model::BootPoint &bp, const CCtVec &x)
{
    const Boot *b = bp.b.get();
    const size_t B = x.size();
    const int N = c->N, L = b->level_top;
    const std::vector<const EvalKey *> &evk = bt->evk;
    Owned r;
    for (size_t q = 0; q < B; q++) {   // boost and ModRaise
        std::unique_ptr<Ciphertext> x0(ct_drop(c, x[q], 0));
        k::mul_scalar_mont(c, x0->data.u(), x0->data.u(), b->boost_mont.u(), 2, c->qmap(0, 0, 1));
        DevMem coef(c, (size_t)2 * N * 8);
        std::vector<k::NttLimb> inv = {{x0->c0(), coef.u(), 0, nullptr, nullptr},
                                       {x0->c1(), coef.u() + N, 0, nullptr, nullptr}};
        k::ntt_run(c, inv, true, nullptr);
        std::unique_ptr<Ciphertext> y(new_ct(c, L, (double)c->primes[0]));
        k::mod_raise(c, y->data.u(), coef.u(), (size_t)N, 2, L + 1, c->qmap(L));
        k::ntt_fwd(c, y->data.u(), 2 * (L + 1), c->qmap(L, 0, L + 1));
        r.v.push_back(std::move(y));
    }
    for (int st : b->subsum_steps) {   // SubSum
        Owned rr = rotate_b(c, evk, r.craw(), {st});
        r = add_b(c, r.craw(), rr.craw());
    }
    Owned y = matvec_b(c, bt, b->cts_a.get(), r.craw());   // CoeffToSlot: C + conj(C)
    r = Owned();
    {
        Owned yc = galois_b(c, evk, y.craw(), {2ull * N - 1});
        y = add_b(c, y.craw(), yc.craw());
    }
    for (int i = 1; i < b->cts_levels; i++) y = rescale_b(c, y.craw());
    for (auto &p : y.v)
        HCHECK(p->scale == b->s_cts && p->level == b->plan->in_level, HELRM_E_SCALE,
               "internal: CoeffToSlot ended on another scale or level");
    y = add_int_b(c, y.craw(), b->c_shift);   // EvalMod
    Owned cv;
    for (Ciphertext *p : poly_b(c, evk, y.craw(), *b->plan)) cv.v.emplace_back(p);
    y = Owned();
    for (int i = 0; i < b->r; i++) {
        cv = square_b(c, evk, cv.craw());
        cv = add_b(c, cv.craw(), cv.craw());
        cv = add_int_b(c, cv.craw(), b->c_double[i]);
    }
    for (auto &p : cv.v)
        HCHECK(p->level == b->level_stc && p->scale == b->s_eval, HELRM_E_LEVEL,
               "internal: EvalMod ended on another level or scale");
    Owned z = matvec_b(c, bt, b->stc.get(), cv.craw());   // SlotToCoeff
    Owned o;
    for (size_t q = 0; q < B; q++) {
        z.v[q]->scale = b->out_scale(x[q]->scale);
        o.v.emplace_back(ct_drop(c, z.v[q].get(), bp.lvl_next));
    }
    return o;
}

std::vector<Ciphertext *> model_infer_batch(Ctx *c, const Batch *bt, const CCtVec &ct_dense, const CCtVec &ct_sel)
{
    const Model *m = bt->model;
    const size_t B = bt->evk.size(), ns = (size_t)m->n_sel();
    HCHECK(ct_dense.size() == B && ct_sel.size() == B * ns, HELRM_E_INVAL, "batch size mismatch");
    for (size_t q = 0; q < B; q++) {
        HCHECK(ct_dense[q]->level == m->lvl_dense, HELRM_E_LEVEL, "ct_dense is not at the model's dense level");
        for (size_t k2 = 0; k2 < ns; k2++)
            HCHECK(ct_sel[q * ns + k2]->level == m->lvl_sel, HELRM_E_LEVEL, "ct_sel is not at the model's selector level");
    }
    // The lookup (selector path) and the bottom MLP (dense path) are
    // independent until z = h + e: the lookup is enqueued on a second stream
    // and overlaps the bottom MLP, then the context's stream joins it.
    const std::vector<PtMatrix *> mats = m->emb_mats();
    Owned e, h;
    Fork branch(c);
    branch.run([&] {
        // one product per selector ciphertext (ct_sel is query-major); the
        // chunks of one shape share their giant steps (matvec_sum_b), and the
        // groups, in order of first appearance, are added in order
        std::vector<std::vector<size_t>> groups;
        for (size_t k2 = 0; k2 < ns; k2++) {
            bool placed = false;
            for (auto &grp : groups)
                if (same_shape(mats[grp[0]], mats[k2])) {
                    grp.push_back(k2);
                    placed = true;
                    break;
                }
            if (!placed) groups.push_back({k2});
        }
        bool first = true;
        for (auto &grp : groups) {
            std::vector<const PtMatrix *> ms;
            std::vector<CCtVec> xs;
            for (size_t k2 : grp) {
                ms.push_back(mats[k2]);
                CCtVec sk2;
                for (size_t q = 0; q < B; q++) sk2.push_back(ct_sel[q * ns + k2]);
                xs.push_back(sk2);
            }
            Owned t = matvec_sum_b(c, bt, ms, xs);
            e = first ? std::move(t) : add_b(c, e.craw(), t.craw());
            first = false;
        }
    });
    CCtVec x = ct_dense;
    Owned hb;
    for (size_t i = 0; i < m->bottom.size(); i++) {
        if (m->boot_b[i].b) {
            hb = boot_all(c, bt, m->boot_b[i], x);
            x = hb.craw();
        }
        h = dense_layer_b(c, bt, m->bottom[i], x);
        x = h.craw();
    }
    hb = Owned();
    branch.join();
    Owned z = add_b(c, h.craw(), e.craw());
    h = Owned();
    e = Owned();
    Owned y;
    if (m->interaction == 0) {
        z = add_pt_b(c, z.craw(), m->ones.get());
        if (m->boot_z.b) z = boot_all(c, bt, m->boot_z, z.craw());
        y = dot_interaction_b(c, bt, m, z.craw());
    } else {
        y = std::move(z);
        if (m->boot_z.b) y = boot_all(c, bt, m->boot_z, y.craw());
    }
    for (size_t i = 0; i < m->top.size(); i++) {
        if (m->boot_t[i].b) y = boot_all(c, bt, m->boot_t[i], y.craw());
        y = dense_layer_b(c, bt, m->top[i], y.craw());
    }
    std::vector<Ciphertext *> out;
    for (auto &p : y.v) out.push_back(p.release());
    return out;
}

// The batch's server path through a CUDA graph.  The first call allocates
// fixed input and output ciphertexts, copies the inputs in, and captures
// model_infer_batch on them (its temporaries become allocation and free nodes
// of the graph, and the logits are copied to the fixed outputs inside it);
// every call then copies its inputs in, launches the graph and copies the
// logits out into new ciphertexts.  The launches, their order and their
// arithmetic are those of the eager path, so the results are identical.
std::vector<Ciphertext *> model_infer_batch_graph(Ctx *c, Batch *bt, const CCtVec &ct_dense, const CCtVec &ct_sel)
{
    const size_t B = bt->evk.size();
    const Model *m = bt->model;
    const size_t S = B * (size_t)m->n_sel();   // ct_sel is query-major, n_sel per query
    HCHECK(ct_dense.size() == B && ct_sel.size() == S, HELRM_E_INVAL, "batch size mismatch");
    HCHECK(!c->prof_on, HELRM_E_INVAL, "kernel profiling cannot be recorded inside a graph");
    for (size_t q = 0; q < B; q++)
        HCHECK(ct_dense[q]->level == m->lvl_dense, HELRM_E_LEVEL, "ct_dense is not at the model's dense level");
    for (size_t r = 0; r < S; r++)
        HCHECK(ct_sel[r]->level == m->lvl_sel, HELRM_E_LEVEL, "ct_sel is not at the model's selector level");
    auto copy_in = [&] {
        for (size_t q = 0; q < B; q++) {
            HCHECK(ct_dense[q]->scale == bt->g_dense[q]->scale, HELRM_E_SCALE, "input scales differ from the captured ones");
            k::copy(c, bt->g_dense[q]->data.u(), ct_dense[q]->data.u(), bt->g_dense[q]->data.bytes / 8);
        }
        for (size_t r = 0; r < S; r++) {
            HCHECK(ct_sel[r]->scale == bt->g_sel[r]->scale, HELRM_E_SCALE, "input scales differ from the captured ones");
            k::copy(c, bt->g_sel[r]->data.u(), ct_sel[r]->data.u(), bt->g_sel[r]->data.bytes / 8);
        }
    };
    if (!bt->exec) {
        for (size_t q = 0; q < B; q++) bt->g_dense.emplace_back(new_ct(c, m->lvl_dense, ct_dense[q]->scale));
        for (size_t r = 0; r < S; r++) bt->g_sel.emplace_back(new_ct(c, m->lvl_sel, ct_sel[r]->scale));
        copy_in();
        // the output buffers and scales come from one eager run on the fixed inputs
        Owned probe;
        {
            std::vector<Ciphertext *> y = model_infer_batch(c, bt, [&] { CCtVec v; for (auto &p : bt->g_dense) v.push_back(p.get()); return v; }(),
                                                            [&] { CCtVec v; for (auto &p : bt->g_sel) v.push_back(p.get()); return v; }());
            for (auto *p : y) probe.v.emplace_back(p);
        }
        for (size_t q = 0; q < B; q++) bt->g_out.emplace_back(new_ct(c, probe.v[q]->level, probe.v[q]->scale));
        probe = Owned();
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        if (!bt->gstream) {
            CUDA_CHECK(cudaStreamCreateWithFlags(&bt->gstream, cudaStreamNonBlocking));
            CUDA_CHECK(cudaEventCreateWithFlags(&bt->ev_in, cudaEventDisableTiming));
            CUDA_CHECK(cudaEventCreateWithFlags(&bt->ev_out, cudaEventDisableTiming));
        }
        c->side_of(bt->gstream);   // the branch stream of the capture exists before it opens
        const cudaStream_t home = c->stream;
        cudaGraph_t g = nullptr;
        CUDA_CHECK(cudaStreamBeginCapture(bt->gstream, cudaStreamCaptureModeThreadLocal));
        c->stream = bt->gstream;   // everything the path enqueues goes into the capture
        c->capturing = true;       // allocations become graph nodes (no side pool)
        try {
            CCtVec d, s;
            for (auto &p : bt->g_dense) d.push_back(p.get());
            for (auto &p : bt->g_sel) s.push_back(p.get());
            std::vector<Ciphertext *> y = model_infer_batch(c, bt, d, s);
            Owned yo;
            for (auto *p : y) yo.v.emplace_back(p);
            for (size_t q = 0; q < B; q++) k::copy(c, bt->g_out[q]->data.u(), yo.v[q]->data.u(), yo.v[q]->data.bytes / 8);
        } catch (...) {
            c->stream = home;
            c->capturing = false;
            cudaStreamEndCapture(bt->gstream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            throw;
        }
        c->stream = home;
        c->capturing = false;
        CUDA_CHECK(cudaStreamEndCapture(bt->gstream, &g));
        cudaError_t e = cudaGraphInstantiate(&bt->exec, g, 0);
        cudaGraphDestroy(g);
        CUDA_CHECK(e);
    } else {
        copy_in();
    }
    // the graph's stream follows the context stream's input copies, and the
    // context stream follows the graph
    CUDA_CHECK(cudaEventRecord(bt->ev_in, c->stream));
    CUDA_CHECK(cudaStreamWaitEvent(bt->gstream, bt->ev_in, 0));
    CUDA_CHECK(cudaGraphLaunch(bt->exec, bt->gstream));
    CUDA_CHECK(cudaEventRecord(bt->ev_out, bt->gstream));
    CUDA_CHECK(cudaStreamWaitEvent(c->stream, bt->ev_out, 0));
    std::vector<Ciphertext *> out;
    for (size_t q = 0; q < B; q++) {
        Ciphertext *o = new_ct(c, bt->g_out[q]->level, bt->g_out[q]->scale);
        k::copy(c, o->data.u(), bt->g_out[q]->data.u(), o->data.bytes / 8);
        out.push_back(o);
    }
    return out;
}

void batch_set_graph(Batch *b, bool on) { b->use_graph = on; }
bool batch_uses_graph(const Batch *b) { return b->use_graph; }
size_t batch_size(const Batch *b) { return b->evk.size(); }
void batch_destroy(Batch *b) { delete b; }
const EvalKey *batch_evk(const Batch *b, size_t q) { return b->evk[q]; }
const Model *batch_model(const Batch *b) { return b->model; }
Ctx *batch_ctx(const Batch *b) { return b->ctx; }

}  // namespace helrm
