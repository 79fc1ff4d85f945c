// kernels.cu -- the device kernels other than the NTT.
//
//  * limb-wise modular arithmetic (add, sub, products in Montgomery form);
//  * fast base conversion (ModUp / ModDown): y_k = sum_s [x_s Qhat_s^-1]_{q_s}
//    (Qhat_s mod p_k) mod p_k, one 128-bit accumulator and one REDC per output;
//  * the fused Galois automorphism + key-switching inner product: for every
//    output word, gather the permuted digit words, multiply by the key words
//    (Montgomery form) and accumulate all digits in 128 bits;
//  * the BSGS multiply-accumulate over QP: inner_g = sum_b diag'_{g,b} * baby_b
//    with the baby-step tile held in shared memory for all giant steps, so every
//    diagonal and every baby step is read from HBM exactly once;
//  * the rescale helper (centred remainder of the dropped limb);
//  * ChaCha20 (RFC 8439) keystream samplers for keys and encryption noise;
//  * the FP64 FFT used by the CKKS encoder and decoder.
#include <cmath>

#include "core.cuh"

#define LAUNCHED(c)                     \
    do {                                \
        (c)->launches++;                \
        CUDA_CHECK(cudaGetLastError()); \
    } while (0)

namespace helrm {
namespace {

constexpr int TPB = 256;

inline unsigned grid_for(size_t n, int tpb = TPB)
{
    size_t g = (n + tpb - 1) / tpb;
    return (unsigned)std::min<size_t>(g, 152 * 64);
}

enum Op { OP_ADD, OP_SUB, OP_NEG, OP_MULM, OP_MULP, OP_TOMONT, OP_FROMMONT };

__global__ void k_binop(u64 *__restrict__ out, const u64 *__restrict__ a, const u64 *__restrict__ b,
                        int logN, size_t total, const PrimeInfo *__restrict__ pinfo, LimbMap map, int op)
{
    pdl_begin();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const PrimeInfo pi = pinfo[map.pid((int)(idx >> logN))];
        u64 x = a[idx], r;
        switch (op) {
        case OP_ADD: r = add_mod(x, b[idx], pi.q); break;
        case OP_SUB: r = sub_mod(x, b[idx], pi.q); break;
        case OP_NEG: r = x ? pi.q - x : 0; break;
        case OP_MULM: r = mont_mul(x, b[idx], pi.q, pi.qinv); break;
        case OP_MULP: r = mul_mod(x, b[idx], pi.q, pi.qinv, pi.r2); break;
        case OP_FROMMONT: r = redc(0, x, pi.q, pi.qinv); break;
        default: r = mont_mul(x, pi.r2, pi.q, pi.qinv); break;   // OP_TOMONT
        }
        out[idx] = r;
    }
}

__global__ void k_tensor(u64 *__restrict__ d, const u64 *__restrict__ a0, const u64 *__restrict__ a1,
                         const u64 *__restrict__ b0, const u64 *__restrict__ b1, int logN, size_t total,
                         const PrimeInfo *__restrict__ pinfo, LimbMap map, int accumulate)
{
    pdl_begin();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const PrimeInfo pi = pinfo[map.pid((int)(idx >> logN))];
        const u64 x0 = a0[idx], x1 = a1[idx], y0 = b0[idx], y1 = b1[idx];
        // REDC gives (sum) R^-1; one more product by R^2 (Montgomery) restores the value
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

// out = a * s[pid]  or  out = (a - b) * s[pid], s in Montgomery form indexed by prime id
__global__ void k_scalar(u64 *__restrict__ out, const u64 *__restrict__ a, const u64 *__restrict__ b,
                         const u64 *__restrict__ scal, int logN, size_t total,
                         const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    pdl_begin();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int pid = map.pid((int)(idx >> logN));
        const PrimeInfo pi = pinfo[pid];
        u64 x = a[idx];
        if (b) x = sub_mod(x, b[idx], pi.q);
        out[idx] = mont_mul(x, scal[pid], pi.q, pi.qinv);
    }
}

__global__ void k_add_scalar(u64 *__restrict__ out, const u64 *__restrict__ a, const u64 *__restrict__ scal,
                             int logN, size_t total, const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    pdl_begin();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int pid = map.pid((int)(idx >> logN));
        out[idx] = add_mod(a[idx], scal[pid], pinfo[pid].q);
    }
}

// blockIdx.y = polynomial p: out + p total <- in + p N (one launch for several)
__global__ void k_from_signed(u64 *__restrict__ out, const i64 *__restrict__ in, int logN, size_t total,
                              const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    pdl_begin();
    const size_t N = (size_t)1 << logN;
    out += blockIdx.y * total;
    in += blockIdx.y * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const u64 q = pinfo[map.pid((int)(idx >> logN))].q;
        i64 v = in[idx & (N - 1)];
        u64 m = (u64)(v < 0 ? -v : v) % q;
        out[idx] = (v < 0 && m) ? q - m : m;
    }
}

// ------------------------------------------------- automorphism + key inner product
// NTT-domain Galois map for the bit-reversed order: slot i holds a(psi^(2x+1)),
// x = brv(i); X -> X^k sends it to the slot of exponent (2x+1)k.
__device__ __forceinline__ int auto_src(int i, int logN, u64 galois)
{
    const u32 x = __brev((u32)i) >> (32 - logN);
    const u64 e = ((2ull * x + 1) * galois) & ((2ull << logN) - 1);
    return (int)(__brev((u32)((e - 1) >> 1)) >> (32 - logN));
}

// DN > 0: the digit count as a constant (every load of a word issued before
// its products); DN = 0 takes dnum_rt.
template <int DN>
__global__ void k_ks_inner(u64 *__restrict__ out, const u64 *__restrict__ dig, int dnum_rt,
                           const u64 *__restrict__ key, int kl, int level, int L, int K, int logN, u64 galois,
                           const u64 *__restrict__ c0, const u64 *__restrict__ pmod,
                           const u64 *__restrict__ bq, int accumulate, const PrimeInfo *__restrict__ pinfo)
{
    pdl_begin();
    const int dnum = DN > 0 ? DN : dnum_rt;
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
        const int src = galois == 1 ? i : auto_src(i, logN, galois);
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

__global__ void k_automorphism(u64 *__restrict__ out, const u64 *__restrict__ in, int logN, size_t total,
                               u64 galois)
{
    pdl_begin();
    const size_t N = (size_t)1 << logN;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t base = idx & ~(N - 1);
        out[idx] = in[base + auto_src((int)(idx & (N - 1)), logN, galois)];
    }
}

// --------------------------------------------------------------- BSGS MAC
// One CTA = TC coefficients of one limb.  The n1 baby steps (two polys each)
// of that tile live in shared memory; the CTA then streams every diagonal of
// every giant step once and writes inner_g for all g.
constexpr int MAC_TC = 128;
__global__ void __launch_bounds__(MAC_TC) k_bsgs_mac(u64 *__restrict__ inner, const u64 *__restrict__ baby,
                                                     const u64 *const *__restrict__ diag,
                                                     const int *__restrict__ gb, int n1, int n2, int nl,
                                                     int logN, const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    pdl_begin();
    extern __shared__ u64 sb[];   // [n1][2][MAC_TC]
    const size_t N = (size_t)1 << logN;
    const int l = blockIdx.y;
    const int i = blockIdx.x * MAC_TC + threadIdx.x;
    const PrimeInfo pi = pinfo[map.pid(l)];
    const size_t plane = (size_t)nl * N;
    for (int b = 0; b < n1; b++) {
        const u64 *bb = baby + (size_t)b * 2 * plane + (size_t)l * N + i;
        sb[(2 * b) * MAC_TC + threadIdx.x] = bb[0];
        sb[(2 * b + 1) * MAC_TC + threadIdx.x] = bb[plane];
    }
    // (no __syncthreads needed: every thread reads back only its own column)
    for (int g = 0; g < n2; g++) {
        Acc128 a0, a1;
        bool any = false;
        for (int b = 0; b < n1; b++) {
            const int di = gb[g * n1 + b];
            if (di < 0) continue;
            any = true;
            const u64 d = diag[di][(size_t)l * N + i];
            a0.mac(sb[(2 * b) * MAC_TC + threadIdx.x], d, pi.q);
            a1.mac(sb[(2 * b + 1) * MAC_TC + threadIdx.x], d, pi.q);
        }
        if (!any) continue;
        u64 *o = inner + (size_t)g * 2 * plane + (size_t)l * N + i;
        o[0] = a0.reduce_long(pi.q, pi.qinv, pi.rmod);
        o[plane] = a1.reduce_long(pi.q, pi.qinv, pi.rmod);
    }
}

// ------------------------------------------------------------------ rescale
// tab: [nP] q_l^-1 (Montgomery, by prime id), [nP] q_l mod q_i, [2 nP] q_l.
__global__ void k_rescale_spread(u64 *__restrict__ out, const u64 *__restrict__ last, const u64 *__restrict__ tab,
                                 int nP, int logN, size_t total, const PrimeInfo *__restrict__ pinfo)
{
    pdl_begin();
    const size_t N = (size_t)1 << logN;
    const u64 ql = tab[2 * nP];
    const u64 half = (ql - 1) >> 1;
    out += blockIdx.y * total;   // poly blockIdx.y: [level][N] from its own last limb
    last += blockIdx.y * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx >> logN);
        const u64 q = pinfo[l].q;
        u64 x = last[idx & (N - 1)];
        u64 xm = x < q ? x : x % q;
        // centred remainder r = x - q_l when x > (q_l - 1)/2
        out[idx] = x <= half ? xm : sub_mod(xm, tab[nP + l], q);
    }
}

__global__ void k_check_range(const u64 *__restrict__ d, int logN, size_t total, const PrimeInfo *__restrict__ pinfo,
                              LimbMap map, int *flag)
{
    pdl_begin();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x)
        if (d[idx] >= pinfo[map.pid((int)(idx >> logN))].q) *flag = 1;
}

// ---------------------------------------------------------------- ChaCha20
__device__ __forceinline__ u32 rotl32(u32 x, int r) { return __funnelshift_l(x, x, r); }
#define QR(a, b, c, d)                 \
    a += b; d ^= a; d = rotl32(d, 16); \
    c += d; b ^= c; b = rotl32(b, 12); \
    a += b; d ^= a; d = rotl32(d, 8);  \
    c += d; b ^= c; b = rotl32(b, 7);

// RFC 8439 Sec. 2.3: constants | key (seed LE, then zeros) | counter | nonce.
__device__ void chacha_block(u64 seed, u32 purpose, u64 index, u32 counter, u32 out[16])
{
    u32 s[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                 (u32)seed, (u32)(seed >> 32), 0, 0, 0, 0, 0, 0,
                 counter, purpose, (u32)index, (u32)(index >> 32)};
    u32 x[16];
#pragma unroll
    for (int i = 0; i < 16; i++) x[i] = s[i];
#pragma unroll
    for (int r = 0; r < 10; r++) {
        QR(x[0], x[4], x[8], x[12]);
        QR(x[1], x[5], x[9], x[13]);
        QR(x[2], x[6], x[10], x[14]);
        QR(x[3], x[7], x[11], x[15]);
        QR(x[0], x[5], x[10], x[15]);
        QR(x[1], x[6], x[11], x[12]);
        QR(x[2], x[7], x[8], x[13]);
        QR(x[3], x[4], x[9], x[14]);
    }
#pragma unroll
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

__global__ void k_chacha_words(u32 *out, u64 seed, u32 purpose, u64 index, u64 first_word, u64 n_words)
{
    pdl_begin();
    const u64 b0 = first_word / 16, b1 = (first_word + n_words + 15) / 16;
    for (u64 b = b0 + blockIdx.x * (u64)blockDim.x + threadIdx.x; b < b1; b += (u64)gridDim.x * blockDim.x) {
        u32 w[16];
        chacha_block(seed, purpose, index, (u32)b, w);
        for (int k2 = 0; k2 < 16; k2++) {
            u64 pos = b * 16 + k2;
            if (pos >= first_word && pos < first_word + n_words) out[pos - first_word] = w[k2];
        }
    }
}

// uniform mod q: coefficient t = gid * N + i takes words 4t..4t+3 as (lo, hi)
__global__ void k_uniform(u64 *out, u64 seed, u32 purpose, u64 index, int logN, int n_limbs,
                          const int *__restrict__ limb_pid, const int *__restrict__ limb_gid,
                          const PrimeInfo *__restrict__ pinfo)
{
    pdl_begin();
    const u64 N = 1ull << logN;
    const u64 per = N / 4;
    const u64 total = per * n_limbs;
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < total; t += (u64)gridDim.x * blockDim.x) {
        const int l = (int)(t / per);
        const u64 i4 = t % per;
        const u64 q = pinfo[limb_pid[l]].q;
        const u64 blk = (u64)limb_gid[l] * per + i4;
        u32 w[16];
        chacha_block(seed, purpose, index, (u32)blk, w);
        for (int c = 0; c < 4; c++) {
            u64 lo = (u64)w[4 * c] | ((u64)w[4 * c + 1] << 32);
            u64 hi = (u64)w[4 * c + 2] | ((u64)w[4 * c + 3] << 32);
            u128 v = ((u128)hi << 64) | lo;
            out[(u64)l * N + 4 * i4 + c] = (u64)(v % q);
        }
    }
}

__global__ void k_ternary(i64 *out, u64 seed, u32 purpose, u64 index, int N)
{
    pdl_begin();
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 16; b += gridDim.x * blockDim.x) {
        u32 w[16];
        chacha_block(seed, purpose, index, (u32)b, w);
        for (int k2 = 0; k2 < 16; k2++) out[16 * b + k2] = (i64)(w[k2] & 1) - (i64)((w[k2] >> 1) & 1);
    }
}

__global__ void k_cbd21(i64 *out, u64 seed, u32 purpose, u64 index, int N)
{
    pdl_begin();
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 8; b += gridDim.x * blockDim.x) {
        u32 w[16];
        chacha_block(seed, purpose, index, (u32)b, w);
        for (int c = 0; c < 8; c++) {
            u64 x = (u64)w[2 * c] | ((u64)w[2 * c + 1] << 32);
            const u64 m = (1ull << 21) - 1;
            out[8 * b + c] = (i64)__popcll(x & m) - (i64)__popcll((x >> 21) & m);
        }
    }
}

// Sparse ternary secret: exactly h coefficients in {-1, +1}.  Stream word i
// (i < N) is the priority of coefficient i, word N + i its sign (bit 0: 0 ->
// +1, 1 -> -1); the h coefficients with the smallest (priority, i) pairs are
// non-zero.  One CTA of SPARSE_T threads: the 2N words go to `words` (global
// scratch), a bisection over the 32-bit values finds the h-th smallest
// priority T, every coefficient below T is taken and, of those equal to T,
// the ones with the smallest positions (a block-wide prefix over contiguous
// chunks of SPARSE_T-th of the positions each).
constexpr int SPARSE_T = 1024;
__device__ int block_sum_int(int v, int *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    return s;
}
__global__ void __launch_bounds__(SPARSE_T) k_sparse_ternary(i64 *out, u32 *words, u64 seed, u32 purpose, int N,
                                                             int h)
{
    pdl_begin();
    __shared__ int red[32];
    __shared__ int pre[SPARSE_T];
    const int t = threadIdx.x, T = blockDim.x, per = N / T;
    for (int b = t; b < 2 * N / 16; b += T) {
        u32 w[16];
        chacha_block(seed, purpose, 0, (u32)b, w);
        for (int k2 = 0; k2 < 16; k2++) words[16 * b + k2] = w[k2];
    }
    __syncthreads();
    const u32 *pr = words + (size_t)t * per;
    // smallest v with #{priority <= v} >= h
    u32 lo = 0, hi = 0xffffffffu;
    while (lo < hi) {
        const u32 mid = lo + ((hi - lo) >> 1);
        int cnt = 0;
        for (int i = 0; i < per; i++) cnt += pr[i] <= mid;
        if (block_sum_int(cnt, red) >= h)
            hi = mid;
        else
            lo = mid + 1;
    }
    int lt = 0, eq = 0;
    for (int i = 0; i < per; i++) {
        lt += pr[i] < lo;
        eq += pr[i] == lo;
    }
    const int need = h - block_sum_int(lt, red);   // how many of the ties are taken, by position
    pre[t] = eq;
    __syncthreads();
    int rank = 0;
    for (int w = 0; w < t; w++) rank += pre[w];
    for (int i = 0; i < per; i++) {
        const int pos = t * per + i;
        bool take = pr[i] < lo;
        if (pr[i] == lo) take = rank++ < need;
        out[pos] = take ? ((words[N + pos] & 1u) ? -1 : 1) : 0;
    }
}

// An encryption's three noise polynomials in one launch (blockIdx.y): v
// ternary from stream pv into out[0..N), e0 and e1 CBD(21) from streams pe0,
// pe1 into out[N..2N) and out[2N..3N); the same words as k_ternary / k_cbd21.
__global__ void k_enc_noise(i64 *out, u64 seed, u32 pv, u32 pe0, u32 pe1, int N)
{
    pdl_begin();
    const int y = blockIdx.y;
    i64 *o = out + (size_t)y * N;
    if (y == 0) {
        for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 16; b += gridDim.x * blockDim.x) {
            u32 w[16];
            chacha_block(seed, pv, 0, (u32)b, w);
            for (int k2 = 0; k2 < 16; k2++) o[16 * b + k2] = (i64)(w[k2] & 1) - (i64)((w[k2] >> 1) & 1);
        }
        return;
    }
    const u32 purpose = y == 1 ? pe0 : pe1;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < N / 8; b += gridDim.x * blockDim.x) {
        u32 w[16];
        chacha_block(seed, purpose, 0, (u32)b, w);
        for (int c = 0; c < 8; c++) {
            u64 x = (u64)w[2 * c] | ((u64)w[2 * c + 1] << 32);
            const u64 m = (1ull << 21) - 1;
            o[8 * b + c] = (i64)__popcll(x & m) - (i64)__popcll((x >> 21) & m);
        }
    }
}

// c0 = v pk0 + e0 + m, c1 = v pk1 + e1 (v, pk Montgomery products; the adds in
// this order), over the n limbs of `total` words
__global__ void k_enc_combine(u64 *__restrict__ c0, u64 *__restrict__ c1, const u64 *__restrict__ v,
                              const u64 *__restrict__ e0, const u64 *__restrict__ e1, const u64 *__restrict__ m,
                              const u64 *__restrict__ pk0, const u64 *__restrict__ pk1, int logN, size_t total,
                              const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    pdl_begin();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const PrimeInfo pi = pinfo[map.pid((int)(idx >> logN))];
        const u64 x = v[idx];
        c0[idx] = add_mod(add_mod(mont_mul(x, pk0[idx], pi.q, pi.qinv), e0[idx], pi.q), m[idx], pi.q);
        c1[idx] = add_mod(mont_mul(x, pk1[idx], pi.q, pi.qinv), e1[idx], pi.q);
    }
}

// ------------------------------------------------------------- FP64 FFT
// The N-point DFT X_k = sum_n x_n e^{-+2 pi i n k / N} (- forward, + inverse)
// as a four-step FFT in two launches: N = R C, n = C n1 + n2, k = k1 + R k2.
// Column pass (COLS): for each n2 the R-point DFT over n1, times e^{-+2 pi i
// n2 k1 / N}, stored at k1 C + n2; row pass: for each k1 the C-point DFT over
// n2, stored at k1 + R k2.  A CTA takes G sub-transforms of P points (P = R or
// C), loads them coalesced, runs the log2 P radix-2 Stockham stages in shared
// memory (one butterfly per thread per stage) and stores them coalesced.
// tw[t] = e^{-2 pi i t / N}, t < N/2.
template <bool COLS>
__global__ void k_fft4(const double2 *__restrict__ x, double2 *__restrict__ y, int logN, int logR, int logP,
                       const double2 *__restrict__ tw, int inverse)
{
    pdl_begin();
    extern __shared__ double2 fsm[];
    const int N = 1 << logN, R = 1 << logR, C = N >> logR, P = 1 << logP;
    const int G = (2 * blockDim.x) >> logP;          // sub-transforms per CTA
    double2 *b0 = fsm, *b1 = fsm + G * P;
    const int base = blockIdx.x * G;                 // first column (COLS) or row
    for (int e = threadIdx.x; e < G * P; e += blockDim.x) {
        if (COLS) {
            const int g = e % G, n1 = e / G;
            b0[g * P + n1] = x[(size_t)n1 * C + base + g];
        } else {
            const int g = e >> logP, n2 = e & (P - 1);
            b0[e] = x[(size_t)(base + g) * C + n2];
        }
    }
    __syncthreads();
    const int half = P / 2, g = threadIdx.x / half, idx = threadIdx.x % half;
    double2 *in = b0, *out = b1;
    for (int s = 0; s < logP; s++) {
        const int m = 1 << s, l = P >> (s + 1);
        const int j = idx >> s, kk = idx & (m - 1);
        double2 w = tw[(size_t)j * m << (logN - logP)];
        if (inverse) w.y = -w.y;
        const double2 c0 = in[g * P + kk + j * m], c1 = in[g * P + kk + j * m + l * m];
        const double2 d = make_double2(c0.x - c1.x, c0.y - c1.y);
        out[g * P + kk + 2 * j * m] = make_double2(c0.x + c1.x, c0.y + c1.y);
        out[g * P + kk + 2 * j * m + m] = make_double2(w.x * d.x - w.y * d.y, w.x * d.y + w.y * d.x);
        __syncthreads();
        double2 *t = in;
        in = out;
        out = t;
    }
    for (int e = threadIdx.x; e < G * P; e += blockDim.x) {
        const int gg = e % G, k = e / G;
        double2 v = in[gg * P + k];
        if (COLS) {   // k = k1, column n2 = base + gg: times e^{-+2 pi i n2 k1 / N}
            const int n2 = base + gg;
            const int t = (int)(((long long)n2 * k) & (N - 1));
            double2 w = t < N / 2 ? tw[t] : make_double2(-tw[t - N / 2].x, -tw[t - N / 2].y);
            if (inverse) w.y = -w.y;
            y[(size_t)k * C + n2] = make_double2(w.x * v.x - w.y * v.y, w.x * v.y + w.y * v.x);
        } else {      // k = k2, row k1 = base + gg
            y[(size_t)(base + gg) + (size_t)R * k] = v;
        }
    }
}

// x[u] = z_{slot(u)} (both u and the conjugate position carry the real slot)
__global__ void k_enc_gather(double2 *x, const double *__restrict__ slots, const int *__restrict__ slot_of,
                             int n_valid, int period, int N)
{
    pdl_begin();
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const int j = slot_of[u] % period;
        x[u] = make_double2(j < n_valid ? slots[j] : 0.0, 0.0);
    }
}

// complex slots: x[u] = z_j at the position of exponent 5^j (u_of_slot[j]),
// conj(z_j) at the position of -5^j
__global__ void k_enc_gather_c(double2 *x, const double *__restrict__ re, const double *__restrict__ im,
                               const int *__restrict__ slot_of, const int *__restrict__ u_of_slot, int n_valid,
                               int period, int N)
{
    pdl_begin();
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const int s = slot_of[u], j = s % period;
        const double a = j < n_valid ? re[j] : 0.0, b = j < n_valid ? im[j] : 0.0;
        x[u] = make_double2(a, u_of_slot[s] == u ? b : -b);
    }
}

// ModRaise: limb 0 of a coefficient-domain polynomial (mod q0), centred in
// (-q0/2, q0/2], as residues of n_limbs limbs; blockIdx.y = polynomial
__global__ void k_mod_raise(u64 *__restrict__ out, const u64 *__restrict__ in0, int logN, size_t total, u64 q0,
                            size_t in_stride, const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    pdl_begin();
    const size_t N = (size_t)1 << logN;
    out += blockIdx.y * total;
    in0 += blockIdx.y * in_stride;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const u64 q = pinfo[map.pid((int)(idx >> logN))].q;
        const u64 v = in0[idx & (N - 1)];
        if (v > (q0 - 1) / 2) {   // negative: v - q0
            const u64 m = (q0 - v) % q;
            out[idx] = m ? q - m : 0;
        } else {
            out[idx] = v % q;
        }
    }
}

// m_k = round_half_away(scale * Re(e^(-i pi k/N) X_k) / N) -> residues
__global__ void k_enc_round(u64 *out, i64 *coeffs, const double2 *__restrict__ X, double scale, int logN,
                            int n_limbs, const PrimeInfo *__restrict__ pinfo, LimbMap map, int *overflow)
{
    pdl_begin();
    const int N = 1 << logN;
    for (int k2 = blockIdx.x * blockDim.x + threadIdx.x; k2 < N; k2 += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi((double)k2 / (double)N, &sn, &cs);
        const double re = (cs * X[k2].x + sn * X[k2].y) / (double)N;
        const double v = scale * re;
        const double r = copysign(floor(fabs(v) + 0.5), v);
        if (!(fabs(r) < 4.6e18)) {
            *overflow = 1;
            continue;
        }
        const i64 m = (i64)r;
        if (coeffs) coeffs[k2] = m;
        const u64 am = (u64)(m < 0 ? -m : m);
        for (int l = 0; l < n_limbs; l++) {
            const u64 q = pinfo[map.pid(l)].q;
            const u64 rr = am % q;
            out[(size_t)l * N + k2] = (m < 0 && rr) ? q - rr : rr;
        }
    }
}

// centred limb-0 coefficients -> y_k = m_k e^(i pi k / N)
__global__ void k_dec_twist(double2 *y, const u64 *__restrict__ m0, u64 q0, int logN)
{
    pdl_begin();
    const int N = 1 << logN;
    for (int k2 = blockIdx.x * blockDim.x + threadIdx.x; k2 < N; k2 += gridDim.x * blockDim.x) {
        const u64 x = m0[k2];
        const double v = x > (q0 - 1) / 2 ? -(double)(q0 - x) : (double)x;
        double sn, cs;
        sincospi((double)k2 / (double)N, &sn, &cs);
        y[k2] = make_double2(v * cs, v * sn);
    }
}

__global__ void k_dec_pick(double *out, const double2 *__restrict__ Y, const int *__restrict__ u_of_slot,
                           double scale, int n)
{
    pdl_begin();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        out[j] = Y[u_of_slot[j]].x / scale;
}

// few slots directly: z_j = (1/scale) sum_k m_k cos(pi t_j k / N), t_j = 2 u_j + 1.
// Pass 1: block b of slot j sums its chunk of k into part[j][b]; pass 2 adds
// the DEC_BLOCKS partials in a fixed order (deterministic).
constexpr int DEC_BLOCKS = 64;
__global__ void k_dec_direct(double *part, const u64 *__restrict__ m0, u64 q0, const int *__restrict__ u_of_slot,
                             int logN)
{
    pdl_begin();
    __shared__ double red[256];
    const int N = 1 << logN;
    const int j = blockIdx.y;
    const u64 t = 2ull * u_of_slot[j] + 1;
    double acc = 0;
    for (int k2 = blockIdx.x * blockDim.x + threadIdx.x; k2 < N; k2 += gridDim.x * blockDim.x) {
        const u64 x = m0[k2];
        const double v = x > (q0 - 1) / 2 ? -(double)(q0 - x) : (double)x;
        const u64 e = (t * (u64)k2) & ((2ull << logN) - 1);
        acc += v * cospi((double)e / (double)N);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[j * DEC_BLOCKS + blockIdx.x] = red[0];
}

__global__ void k_dec_sum(double *out, const double *__restrict__ part, double scale, int n)
{
    pdl_begin();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0;
    for (int b = 0; b < DEC_BLOCKS; b++) s += part[j * DEC_BLOCKS + b];
    out[j] = s / scale;
}

__global__ void k_pack_selector(double *sel, const u64 *__restrict__ idx, const int *__restrict__ tab, int T,
                                int base)
{
    pdl_begin();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        u64 i = idx[t];
        const int rows = tab[3 * t], off = tab[3 * t + 1], nd = tab[3 * t + 2];
        if (i >= (u64)rows) continue;   // out-of-range index: no slot set for this table
        if (nd == 0) {   // a plain one-hot
            sel[off + i] = 1.0;
        } else {
            for (int j = 0; j < nd; j++) {   // little-endian base-p digits, one one-hot each
                sel[off + j * base + (int)(i % (u64)base)] = 1.0;
                i /= (u64)base;
            }
        }
    }
}

}  // namespace

namespace k {

__global__ void k_sigmoid(double *p, const double *__restrict__ x, int n)
{
    pdl_begin();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 1.0 / (1.0 + exp(-x[i]));
}

void sigmoid(Ctx *c, double *d_p, const double *d_x, int n)
{
    launch(c, k_sigmoid, (n + 127) / 128, 128, 0, d_p, d_x, n);
    LAUNCHED(c);
}

void pack_selector(Ctx *c, double *sel, const u64 *d_idx, const int *d_tab, int T, int base, int in_pad)
{
    CUDA_CHECK(cudaMemsetAsync(sel, 0, (size_t)in_pad * 8, c->stream));
    launch(c, k_pack_selector, (T + 127) / 128, 128, 0, sel, d_idx, d_tab, T, base);
    LAUNCHED(c);
}


void copy(Ctx *c, u64 *dst, const u64 *src, size_t n)
{
    if (n) CUDA_CHECK(cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, c->stream));
}
void zero(Ctx *c, u64 *dst, size_t n)
{
    if (n) CUDA_CHECK(cudaMemsetAsync(dst, 0, n * 8, c->stream));
}

static void binop(Ctx *c, u64 *out, const u64 *a, const u64 *b, int n_limbs, LimbMap map, int op)
{
    size_t total = (size_t)n_limbs * c->N;
    if (!total) return;
    KTimer kt(c, "elementwise", (b ? 24.0 : 16.0) * total);
    launch(c, k_binop, grid_for(total), TPB, 0, out, a, b, c->logN, total, c->d_pinfo.as<PrimeInfo>(), map, op);
    LAUNCHED(c);
}
void add(Ctx *c, u64 *o, const u64 *a, const u64 *b, int n, LimbMap m) { binop(c, o, a, b, n, m, OP_ADD); }
void sub(Ctx *c, u64 *o, const u64 *a, const u64 *b, int n, LimbMap m) { binop(c, o, a, b, n, m, OP_SUB); }
void neg(Ctx *c, u64 *o, const u64 *a, int n, LimbMap m) { binop(c, o, a, nullptr, n, m, OP_NEG); }
void mul_mont(Ctx *c, u64 *o, const u64 *a, const u64 *b, int n, LimbMap m) { binop(c, o, a, b, n, m, OP_MULM); }
void mul_plain(Ctx *c, u64 *o, const u64 *a, const u64 *b, int n, LimbMap m) { binop(c, o, a, b, n, m, OP_MULP); }
void to_mont(Ctx *c, u64 *o, const u64 *a, int n, LimbMap m) { binop(c, o, a, nullptr, n, m, OP_TOMONT); }
void from_mont(Ctx *c, u64 *o, const u64 *a, int n, LimbMap m) { binop(c, o, a, nullptr, n, m, OP_FROMMONT); }
void tensor(Ctx *c, u64 *d, const u64 *a0, const u64 *a1, const u64 *b0, const u64 *b1, int n_limbs, LimbMap map,
            bool accumulate)
{
    size_t total = (size_t)n_limbs * c->N;
    KTimer kt(c, "tensor", (accumulate ? 10.0 : 7.0) * 8 * total);
    launch(c, k_tensor, grid_for(total), TPB, 0, d, a0, a1, b0, b1, c->logN, total, c->d_pinfo.as<PrimeInfo>(),
                                                     map, accumulate ? 1 : 0);
    LAUNCHED(c);
}

void mul_scalar_mont(Ctx *c, u64 *out, const u64 *a, const u64 *scal, int n_limbs, LimbMap map)
{
    size_t total = (size_t)n_limbs * c->N;
    if (!total) return;
    KTimer kt(c, "elementwise", 16.0 * total);
    launch(c, k_scalar, grid_for(total), TPB, 0, out, a, nullptr, scal, c->logN, total,
                                                     c->d_pinfo.as<PrimeInfo>(), map);
    LAUNCHED(c);
}
void add_scalar(Ctx *c, u64 *out, const u64 *a, const u64 *scal, int n_limbs, LimbMap map)
{
    const size_t total = (size_t)n_limbs * c->N;
    if (!total) return;
    KTimer kt(c, "elementwise", 16.0 * total);
    launch(c, k_add_scalar, grid_for(total), TPB, 0, out, a, scal, c->logN, total, c->d_pinfo.as<PrimeInfo>(), map);
    LAUNCHED(c);
}
void sub_mul_scalar(Ctx *c, u64 *out, const u64 *a, const u64 *b, const u64 *scal, int n_limbs, LimbMap map)
{
    size_t total = (size_t)n_limbs * c->N;
    if (!total) return;
    KTimer kt(c, "elementwise", 24.0 * total);
    launch(c, k_scalar, grid_for(total), TPB, 0, out, a, b, scal, c->logN, total,
                                                     c->d_pinfo.as<PrimeInfo>(), map);
    LAUNCHED(c);
}
void from_signed(Ctx *c, u64 *out, const i64 *in, int n_limbs, LimbMap map, int n_polys)
{
    size_t total = (size_t)n_limbs * c->N;
    if (!total || n_polys < 1) return;
    launch(c, k_from_signed, dim3(grid_for(total), n_polys), TPB, 0, out, in, c->logN, total,
           c->d_pinfo.as<PrimeInfo>(), map);
    LAUNCHED(c);
}
void sample_enc_noise(Ctx *c, i64 *out3, u64 seed, u32 pv, u32 pe0, u32 pe1)
{
    launch(c, k_enc_noise, dim3(grid_for(c->N / 8), 3), TPB, 0, out3, seed, pv, pe0, pe1, c->N);
    LAUNCHED(c);
}
void enc_combine(Ctx *c, u64 *c0, u64 *c1, const u64 *v, const u64 *e0, const u64 *e1, const u64 *m, const u64 *pk0,
                 const u64 *pk1, int n_limbs, LimbMap map)
{
    size_t total = (size_t)n_limbs * c->N;
    if (!total) return;
    launch(c, k_enc_combine, grid_for(total), TPB, 0, c0, c1, v, e0, e1, m, pk0, pk1, c->logN, total,
           c->d_pinfo.as<PrimeInfo>(), map);
    LAUNCHED(c);
}
void ks_inner_auto(Ctx *c, u64 *out, const u64 *digits, int dnum, const SwitchKey *key, int level, u64 galois,
                   const u64 *c0, const u64 *d_pmod_mont, const u64 *bq, bool accumulate)
{
    HCHECK(key->level >= level, HELRM_E_NOKEY, "switching key generated below the level of its use");
    size_t total = (size_t)(level + 1 + c->K) * c->N;
    // digits once, both key halves once, c0 / bq once (if added), two output polys
    // written (and read, when accumulating)
    KTimer kt(c, "ks_inner_auto", 8.0 * (total * (3.0 * dnum + (accumulate ? 4 : 2) + (bq ? 1 : 0)) +
                                         (c0 ? (double)(level + 1) * c->N : 0.0)));
    using Fn = void (*)(u64 *, const u64 *, int, const u64 *, int, int, int, int, int, u64, const u64 *, const u64 *,
                        const u64 *, int, const PrimeInfo *);
    static const Fn fns[] = {k_ks_inner<0>, k_ks_inner<1>, k_ks_inner<2>, k_ks_inner<3>, k_ks_inner<4>,
                             k_ks_inner<5>, k_ks_inner<6>, k_ks_inner<7>, k_ks_inner<8>, k_ks_inner<9>};
    launch(c, fns[dnum >= 1 && dnum <= 9 ? dnum : 0], grid_for(total), TPB, 0, out, digits, dnum, key->data.u(),
           key->level, level, c->L, c->K,
           c->logN, galois, c0,
                                                 d_pmod_mont, bq, accumulate ? 1 : 0, c->d_pinfo.as<PrimeInfo>());
    LAUNCHED(c);
}
void automorphism(Ctx *c, u64 *out, const u64 *in, int n_limbs, u64 galois)
{
    size_t total = (size_t)n_limbs * c->N;
    if (!total) return;
    KTimer kt(c, "automorphism", 16.0 * total);
    launch(c, k_automorphism, grid_for(total), TPB, 0, out, in, c->logN, total, galois);
    LAUNCHED(c);
}
void bsgs_mac(Ctx *c, u64 *inner, const u64 *baby, int n_baby, const u64 *const *d_diag_ptrs,
              const int *d_gb_index, int n2, int n1, int limbs, LimbMap map)
{
    size_t smem = (size_t)n1 * 2 * MAC_TC * 8;
    // n_baby: number of distinct diagonals (non-zero); babies read once, diagonals once,
    // n2 inner ciphertexts written once
    KTimer kt(c, "bsgs_mac", 8.0 * limbs * c->N * (2.0 * n1 + (double)n_baby + 2.0 * n2));
    HCHECK(smem <= 200 * 1024, HELRM_E_PARAM, "too many baby steps for the MAC tile");
    if (smem > 48 * 1024)
        CUDA_CHECK(cudaFuncSetAttribute(k_bsgs_mac, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(c->N / MAC_TC, limbs);
    launch(c, k_bsgs_mac, grid, MAC_TC, smem, inner, baby, d_diag_ptrs, d_gb_index, n1, n2, limbs, c->logN,
                                                  c->d_pinfo.as<PrimeInfo>(), map);
    LAUNCHED(c);
}
void rescale_spread(Ctx *c, u64 *out, const u64 *last_coef, int level, int n_polys)
{
    size_t total = (size_t)level * c->N;
    if (!total) return;
    KTimer kt(c, "rescale_spread", 8.0 * n_polys * (total + c->N));
    launch(c, k_rescale_spread, dim3(grid_for(total), n_polys), TPB, 0, out, last_coef, c->rescale_table(level), c->nP(),
                                                             c->logN, total, c->d_pinfo.as<PrimeInfo>());
    LAUNCHED(c);
}
void check_range(Ctx *c, const u64 *data, int n_limbs, LimbMap map, int *d_flag)
{
    size_t total = (size_t)n_limbs * c->N;
    launch(c, k_check_range, grid_for(total), TPB, 0, data, c->logN, total, c->d_pinfo.as<PrimeInfo>(), map,
                                                          d_flag);
    LAUNCHED(c);
}
void chacha_words(Ctx *c, u32 *out, u64 seed, u32 purpose, u64 index, u64 first_word, u64 n_words)
{
    u64 blocks = (first_word + n_words + 15) / 16 - first_word / 16;
    launch(c, k_chacha_words, grid_for(blocks), TPB, 0, out, seed, purpose, index, first_word, n_words);
    LAUNCHED(c);
}
void sample_uniform(Ctx *c, u64 *out, u64 seed, u32 purpose, u64 index, int n_limbs, const int *d_limb_pid,
                    const int *d_limb_gid)
{
    size_t total = (size_t)n_limbs * c->N / 4;
    launch(c, k_uniform, grid_for(total), TPB, 0, out, seed, purpose, index, c->logN, n_limbs, d_limb_pid,
                                                      d_limb_gid, c->d_pinfo.as<PrimeInfo>());
    LAUNCHED(c);
}
void sample_ternary(Ctx *c, i64 *out, u64 seed, u32 purpose, u64 index)
{
    launch(c, k_ternary, grid_for(c->N / 16), TPB, 0, out, seed, purpose, index, c->N);
    LAUNCHED(c);
}
void sample_sparse_ternary(Ctx *c, i64 *out, u64 seed, u32 purpose, int h)
{
    HCHECK(h > 0 && h <= c->N, HELRM_E_INVAL, "the secret's Hamming weight must be in [1, N]");
    DevMem words(c, (size_t)2 * c->N * 4);
    const int T = std::min(SPARSE_T, c->N);
    launch(c, k_sparse_ternary, 1, T, 0, out, words.as<u32>(), seed, purpose, c->N, h);
    LAUNCHED(c);
    CUDA_CHECK(cudaStreamSynchronize(c->stream));   // the scratch words are freed on return
}
void mod_raise(Ctx *c, u64 *out, const u64 *in0_coef, size_t in_stride, int n_polys, int n_limbs, LimbMap map)
{
    size_t total = (size_t)n_limbs * c->N;
    launch(c, k_mod_raise, dim3(grid_for(total), n_polys), TPB, 0, out, in0_coef, c->logN, total, c->primes[0],
           in_stride, c->d_pinfo.as<PrimeInfo>(), map);
    LAUNCHED(c);
}
void sample_cbd21(Ctx *c, i64 *out, u64 seed, u32 purpose, u64 index)
{
    launch(c, k_cbd21, grid_for(c->N / 8), TPB, 0, out, seed, purpose, index, c->N);
    LAUNCHED(c);
}

// N-point DFT of buf_a (four-step, k_fft4): the result lands in buf_a again
// (the column pass writes buf_b, the row pass buf_a)
static void fft(Ctx *c, double2 *buf_a, double2 *buf_b, bool inverse, double2 **result)
{
    const int logN = c->logN, logR = logN / 2, logC = logN - logR;
    constexpr int G = 4;   // sub-transforms per CTA
    const double2 *tw = c->d_fft_tw.as<double2>();
    launch(c, k_fft4<true>, (1 << logC) / G, G << (logR - 1), (size_t)2 * G * (8 << logR) * 2, buf_a, buf_b, logN,
           logR, logR, tw, inverse ? 1 : 0);
    LAUNCHED(c);
    launch(c, k_fft4<false>, (1 << logR) / G, G << (logC - 1), (size_t)2 * G * (8 << logC) * 2, buf_b, buf_a, logN,
           logR, logC, tw, inverse ? 1 : 0);
    LAUNCHED(c);
    *result = buf_a;
}

void encode_slots(Ctx *c, u64 *out, const double *d_slots, int n_valid, int period, double scale, int n_limbs,
                  LimbMap map, i64 *d_coeffs_out, const double *d_slots_im)
{
    DevMem a(c, (size_t)c->N * sizeof(double2)), b(c, (size_t)c->N * sizeof(double2));
    KTimer kt(c, "encode_fft", 8.0 * c->N * n_limbs);
    if (d_slots_im)
        launch(c, k_enc_gather_c, grid_for(c->N), TPB, 0, a.as<double2>(), d_slots, d_slots_im,
               c->d_slot_of.as<int>(), c->d_u_of_slot.as<int>(), n_valid, period, c->N);
    else
        launch(c, k_enc_gather, grid_for(c->N), TPB, 0, a.as<double2>(), d_slots, c->d_slot_of.as<int>(), n_valid,
               period, c->N);
    LAUNCHED(c);
    double2 *X;
    fft(c, a.as<double2>(), b.as<double2>(), false, &X);
    launch(c, k_enc_round, grid_for(c->N), TPB, 0, out, d_coeffs_out, X, scale, c->logN, n_limbs,
                                                       c->d_pinfo.as<PrimeInfo>(), map, c->d_err.as<int>());
    LAUNCHED(c);
    // an overflow is reported by the next synchronising call (Ctx::check_device_errors)
}

void decode_limb0(Ctx *c, double *d_out, const u64 *m0, double scale, int n_slots)
{
    const u64 q0 = c->primes[0];
    KTimer kt(c, "decode", 8.0 * c->N);
    if (n_slots <= 16) {
        DevMem part(c, (size_t)n_slots * DEC_BLOCKS * 8);
        launch(c, k_dec_direct, dim3(DEC_BLOCKS, n_slots), 256, 0, part.as<double>(), m0, q0,
                                                                       c->d_u_of_slot.as<int>(), c->logN);
        LAUNCHED(c);
        launch(c, k_dec_sum, 1, 32, 0, d_out, part.as<double>(), scale, n_slots);
        LAUNCHED(c);
        return;
    }
    DevMem a(c, (size_t)c->N * sizeof(double2)), b(c, (size_t)c->N * sizeof(double2));
    launch(c, k_dec_twist, grid_for(c->N), TPB, 0, a.as<double2>(), m0, q0, c->logN);
    LAUNCHED(c);
    double2 *Y;
    fft(c, a.as<double2>(), b.as<double2>(), true, &Y);
    launch(c, k_dec_pick, grid_for(n_slots), TPB, 0, d_out, Y, c->d_u_of_slot.as<int>(), scale, n_slots);
    LAUNCHED(c);
}

}  // namespace k
}  // namespace helrm
