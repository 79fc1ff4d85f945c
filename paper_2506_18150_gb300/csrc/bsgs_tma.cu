// bsgs_tma.cu -- the hoisted baby steps fused into the BSGS multiply-
// accumulate, fed by bulk asynchronous copies (cp.async.bulk + mbarrier).
//
// One CTA owns a tile of T = 256 consecutive coefficients of one limb l of the
// level-ell QP basis and walks the needed baby steps b.  For baby step b it
// needs, per coefficient i of the tile:
//   * the ModUp digits at the Galois source position src(i) (DN words);
//   * key b's two halves at i (2 DN words), and c0 at src(i);
//   * the diagonal words of every giant step g at i (N2 words).
// In the bit-reversed NTT order the automorphism maps an aligned block of 2^m
// consecutive coefficients onto an aligned block of 2^m consecutive
// coefficients (permuted inside), so every one of these is one contiguous
// 2 KB row: a producer lane issues it as a bulk copy into a shared-memory
// stage and the stage's mbarrier counts the bytes in.  With S = 3 stages the
// copies for the next baby steps are in flight while the current one is
// multiplied, so HBM latency is hidden without registers.  Each baby step's
// value (key inner product + P phi(c0)) is reduced and multiplied at once into
// the n2 giant-step accumulators, 64-bit, reduced per product (REDC is linear,
// so the result equals the unfused kernels' bit for bit).
//
// Every wait on an mbarrier is bounded: if a stage does not complete within
// the limit the CTA records HELRM_E_TIMEOUT in the context's error word, waits
// (bounded again) for the copies it issued, and returns.
#include "core.cuh"

namespace helrm {
namespace {

constexpr int T = 256;             // coefficients per tile (= threads per CTA)
constexpr long WAIT_LIMIT = 1L << 24;

__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64 *bar, u32 count)
{
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(u64 *bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64 *bar, u32 parity)
{
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, u32 bytes, u64 *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Source index of slot i under X -> X^galois in the bit-reversed NTT order,
// from xi = 2 brv(i) + 1: only (xi galois) mod 2N matters and 2N <= 2^17, so
// 32-bit arithmetic is exact.
__device__ __forceinline__ int auto_src_x(u32 xi, int logN, u32 galois)
{
    const u32 e = (xi * galois) & ((2u << logN) - 1u);
    return (int)(__brev((e - 1u) >> 1) >> (32 - logN));
}
__device__ __forceinline__ u32 odd_of(int i, int logN) { return 2u * (__brev((u32)i) >> (32 - logN)) + 1u; }

// Per-query operands of one batched launch (kernel parameters).  The batch
// index is the fastest grid dimension, so the CTAs of all queries that work
// on the same tile run together and the diagonal rows they share are read
// from HBM once and served to the others from L2.
constexpr int BQ = 64;
struct TmaQueries {
    u64 *inner[BQ];
    const u64 *dig[BQ];
    const u64 *c0[BQ];
    const u64 *c1[BQ];
};
struct TmaGals {
    u64 gal[64];          // Galois element of baby step b
};

// Stage layout (words): dig[DN][T] | kb[DN][T] | ka[DN][T] | dd[N2][T].  The
// gathered c0 word (L2-resident, one per thread) is not staged: each consumer
// loads it itself one baby step ahead, which keeps the stage smaller.
// Pipeline depth: as many stages (up to 4) as leave two CTAs per SM (at most
// 108 KB of stages per CTA): the consumers stall on stages still in flight
// (the copies' latency under load exceeds two steps of arithmetic), so every
// extra stage the shared memory holds is time the copies get to land.
// With many digits (the 7- to 9-digit key switches at the top of the
// bootstrappable chain) two stages of every row would not fit two CTAs per SM;
// there the diagonal rows stay out of the stage (DD): the consumers read their
// own diagonal words from global memory (coalesced, one word per thread and
// giant step), issued before the key products they then wait behind, and
// the stage keeps the digit and key rows only.
template <int N2, int DN>
struct Stage {
    static constexpr bool DD = 2 * (3 * DN + N2) * T * 8 > 108 * 1024;
    static constexpr int WORDS = (3 * DN + (DD ? 0 : N2)) * T;
    static constexpr int S = (4 * WORDS * 8 <= 108 * 1024) ? 4 : (3 * WORDS * 8 <= 108 * 1024) ? 3 : 2;
};

__device__ __forceinline__ void mbar_arrive(u64 *bar)
{
    asm volatile("mbarrier.arrive.shared.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(u64 *bar, u32 parity)
{
    for (long it = 0; it < WAIT_LIMIT; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Warp-specialised pipeline: warps 0..7 consume (one coefficient per thread),
// warp 8 produces.  full[s] completes when stage s's bytes have landed
// (producer arrive + expect_tx, copies complete_tx); empty[s] completes when
// all 8 consumer warps have read stage s, letting the producer refill it.
constexpr int CONSUMER_WARPS = T / 32;

template <int N2, int DN>
// Two CTAs per SM (2 x 9 warps): an SM partition holds 16K registers and gets
// five of the 18 warps, so a thread may use at most 96 registers.
__global__ void __launch_bounds__(T + 32, 2) k_bsgs_tma(
                                                    const TmaQueries qs, const TmaGals bk,
                                                    const u64 *const *__restrict__ keytab,
                                                    const int *__restrict__ keylv,
                                                    const u64 *const *__restrict__ diag,
                                                    const int *__restrict__ gb, int n1, int level, int L, int K,
                                                    int logN, const u64 *__restrict__ pmod,
                                                    const PrimeInfo *__restrict__ pinfo, int *err)
{
    pdl_begin();
    extern __shared__ __align__(128) u64 smem[];
    constexpr int SW = Stage<N2, DN>::WORDS;
    constexpr int S = Stage<N2, DN>::S;
    constexpr bool DD = Stage<N2, DN>::DD;
    u64 *full = smem + S * SW;        // S mbarriers
    u64 *empty = full + S;            // S mbarriers
    __shared__ int sgb[64 * 8];
    __shared__ int blist[64];         // needed baby steps b >= 1, in order
    __shared__ int nb, need0;
    // per stage, written by the producer before the stage's arrive (so visible
    // to the consumers once the stage completes): the Galois element, the
    // aligned block the gathered rows start at, and which diagonals are present
    __shared__ u32 st_gal[S], st_mask[S];
    __shared__ int st_base[S];
    __shared__ const u64 *s_key[64];   // this query's key of each baby step, and its level
    __shared__ int s_kl[64];
    const int tid = threadIdx.x;
    const size_t N = (size_t)1 << logN;
    const int nl = level + 1 + K;
    const size_t plane = (size_t)nl * N;
    const int qi = blockIdx.x;
    const int l = blockIdx.z;
    const int i0 = blockIdx.y * T;
    u64 *const inner = qs.inner[qi];
    const u64 *const dig = qs.dig[qi];
    const u64 *const c0 = qs.c0[qi];
    const u64 *const c1 = qs.c1[qi];
    const bool qlimb = l <= level;
    const int pid = qlimb ? l : L + 1 + (l - level - 1);

    for (int t = tid; t < n1 * N2; t += blockDim.x) sgb[t] = gb[t];
    for (int t = tid; t < n1; t += blockDim.x) {
        s_key[t] = keytab[(size_t)qi * 64 + t];
        s_kl[t] = keylv[(size_t)qi * 64 + t];
    }
    __syncthreads();
    if (tid == 0) {
        int c = 0;
        for (int b = 1; b < n1; b++) {
            int need = 0;
            for (int g = 0; g < N2; g++) need |= sgb[g * n1 + b] >= 0;
            if (need) blist[c++] = b;
        }
        int n0 = 0;
        for (int g = 0; g < N2; g++) n0 |= sgb[g * n1] >= 0;
        nb = c;
        need0 = n0;
        for (int s = 0; s < S; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CONSUMER_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();   // the last CTA-wide barrier: from here on warps run independently

    if (tid >= T) {
        // ---------------- producer warp
        const int lane = tid & 31;
        int k = 0, s = 0;
        u32 phase = 0;
        bool ok = true;
        const u32 x0 = odd_of(i0, logN);
        for (; k < nb; k++) {
            if (k >= S && !mbar_wait_bounded(&empty[s], phase ^ 1u)) {
                ok = false;
                break;
            }
            const int b = blist[k];
            u64 *st = smem + s * SW;
            const int src_base = auto_src_x(x0, logN, (u32)bk.gal[b]) & ~(T - 1);
            const u64 *key = s_key[b];
            const int kl = s_kl[b], nK = kl + 1 + K, kx = key_limb(pid, kl, L);
            int nd = 0;
            u32 mask = 0;
            for (int g = 0; g < N2; g++)
                if (sgb[g * n1 + b] >= 0) {
                    nd++;
                    mask |= 1u << g;
                }
            if (lane == 0) {
                st_gal[s] = (u32)bk.gal[b];
                st_base[s] = src_base;
                st_mask[s] = mask;
                mbar_arrive_expect_tx(&full[s], (u32)(3 * DN + (DD ? 0 : nd)) * T * 8);
            }
            __syncwarp();
            // rows: DN digit rows, 2 DN key rows, the present diagonal rows (not with DD)
            for (int cidx = lane; cidx < 3 * DN + (DD ? 0 : N2); cidx += 32) {
                const u64 *src = nullptr;
                u64 *dst = nullptr;
                if (cidx < DN) {
                    src = dig + ((size_t)cidx * nl + l) * N + src_base;
                    dst = st + cidx * T;
                } else if (cidx < 2 * DN) {
                    const int j = cidx - DN;
                    src = key + ((size_t)(2 * j) * nK + kx) * N + i0;
                    dst = st + (DN + j) * T;
                } else if (cidx < 3 * DN) {
                    const int j = cidx - 2 * DN;
                    src = key + ((size_t)(2 * j + 1) * nK + kx) * N + i0;
                    dst = st + (2 * DN + j) * T;
                } else {
                    const int g = cidx - 3 * DN;
                    const int di = sgb[g * n1 + b];
                    if (di >= 0) {
                        src = diag[di] + (size_t)l * N + i0;
                        dst = st + (3 * DN + g) * T;
                    }
                }
                if (src) bulk_g2s(dst, src, T * 8, &full[s]);
            }
            __syncwarp();
            if (++s == S) {
                s = 0;
                phase ^= 1u;
            }
        }
        if (!ok && lane == 0) {
            atomicExch(err, (int)HELRM_E_TIMEOUT);
            // let the copies already issued land before the CTA's shared memory goes away
            for (int kk = (k >= S ? k - S : 0); kk < k; kk++) mbar_wait_bounded(&full[kk % S], (u32)((kk / S) & 1));
        }
        return;
    }

    // ---------------- consumer warps: thread tid owns coefficient i0 + tid
    const PrimeInfo pi = pinfo[pid];
    const u64 pm = pmod[pid];
    const int i = i0 + tid;
    const size_t idx = (size_t)l * N + i;
    const int lane = tid & 31;
    Acc128 a0[N2], a1[N2];   // one full product per diagonal word, one REDC at the end
    if (need0) {             // baby 0 = (P c0, P c1): P mod q on the Q limbs, 0 on the P limbs
        const u64 v0 = qlimb ? mont_mul(c0[idx], pm, pi.q, pi.qinv) : 0;
        const u64 v1 = qlimb ? mont_mul(c1[idx], pm, pi.q, pi.qinv) : 0;
#pragma unroll
        for (int g = 0; g < N2; g++) {
            const int di = sgb[g * n1];
            if (di < 0) continue;
            const u64 d = diag[di][idx];
            a0[g].mac(v0, d, pi.q);
            a1[g].mac(v1, d, pi.q);
        }
    }
    const u32 xi = odd_of(i, logN);
    const u64 *c0l = c0 + (size_t)l * N;
    // phi(c0) word of the next baby step, loaded one step ahead (Q limbs only)
    u64 c0_next = (qlimb && nb > 0) ? __ldg(c0l + auto_src_x(xi, logN, (u32)bk.gal[blist[0]])) : 0;
    u32 phase = 0;
    for (int k = 0, s = 0; k < nb; k++) {
        const u64 c0v = c0_next;
        if (qlimb && k + 1 < nb) c0_next = __ldg(c0l + auto_src_x(xi, logN, (u32)bk.gal[blist[k + 1]]));
        if (!mbar_wait_bounded(&full[s], phase)) {
            if (lane == 0) atomicExch(err, (int)HELRM_E_TIMEOUT);
            return;   // no CTA barrier follows, so leaving early cannot deadlock
        }
        const u64 *st = smem + s * SW;
        const u32 mask = st_mask[s];
        const int src_loc = auto_src_x(xi, logN, st_gal[s]) - st_base[s];
        u64 dd_g[DD ? N2 : 1];   // DD: this baby step's diagonal words, loaded before the key products
        if constexpr (DD) {
            const int b = blist[k];
#pragma unroll
            for (int g = 0; g < N2; g++) {
                const int di = sgb[g * n1 + b];
                dd_g[g] = di >= 0 ? __ldg(diag[di] + idx) : 0;
            }
        }
        Acc128 t0, t1;
#pragma unroll
        for (int j = 0; j < DN; j++) {
            const u64 d = st[j * T + src_loc];
            t0.mac(d, st[(DN + j) * T + tid], pi.q);
            t1.mac(d, st[(2 * DN + j) * T + tid], pi.q);
        }
        // + P phi(c0) on the Q limbs: pm = P R mod q, so the same REDC yields it
        if (qlimb) t0.mac(c0v, pm, pi.q);
        const u64 v0 = t0.reduce(pi.q, pi.qinv);
        const u64 v1 = t1.reduce(pi.q, pi.qinv);
        if constexpr (DD) {   // the stage holds no diagonals: release it, then the products
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
            for (int g = 0; g < N2; g++) {
                a0[g].mac(v0, dd_g[g], pi.q);
                a1[g].mac(v1, dd_g[g], pi.q);
            }
        } else if (N2 <= 4) {   // few diagonals: take them into registers and release the stage first
            u64 dd[N2];
#pragma unroll
            for (int g = 0; g < N2; g++) dd[g] = (mask >> g) & 1u ? st[(3 * DN + g) * T + tid] : 0;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
#pragma unroll
            for (int g = 0; g < N2; g++) {
                a0[g].mac(v0, dd[g], pi.q);
                a1[g].mac(v1, dd[g], pi.q);
            }
        } else {         // many: read each as it is used (fewer live registers), then release
#pragma unroll
            for (int g = 0; g < N2; g++) {
                const u64 d = (mask >> g) & 1u ? st[(3 * DN + g) * T + tid] : 0;
                a0[g].mac(v0, d, pi.q);
                a1[g].mac(v1, d, pi.q);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (++s == S) {
            s = 0;
            phase ^= 1u;
        }
    }
#pragma unroll
    for (int g = 0; g < N2; g++) {
        bool any = false;
        for (int b = 0; b < n1; b++) any |= sgb[g * n1 + b] >= 0;
        if (!any) continue;
        u64 *o = inner + (size_t)g * 2 * plane + idx;
        o[0] = a0[g].reduce_long(pi.q, pi.qinv, pi.rmod);   // up to 65 terms
        o[plane] = a1[g].reduce_long(pi.q, pi.qinv, pi.rmod);
    }
}

template <int N2, int DN>
void launch_tma(Ctx *c, const TmaQueries &qs, int nq, const TmaGals &bk, const u64 *const *keytab,
                const int *keylv, const u64 *const *diag, const int *gb, int n1, int level)
{
    constexpr int S = Stage<N2, DN>::S;
    const size_t smem = (size_t)S * Stage<N2, DN>::WORDS * 8 + 2 * S * 8;
    static bool attr_set = false;   // once per instance (also keeps it out of graph captures)
    if (!attr_set) {
        CUDA_CHECK(cudaFuncSetAttribute(k_bsgs_tma<N2, DN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    dim3 grid(nq, c->N / T, level + 1 + c->K);
    launch(c, k_bsgs_tma<N2, DN>, grid, T + 32, smem, qs, bk, keytab, keylv, diag, gb, n1, level, c->L, c->K, c->logN,
           c->d_pmod_mont.u(), c->d_pinfo.as<PrimeInfo>(), c->d_err.as<int>());
}

// The bounded wait of the pipeline on a barrier that no thread ever arrives
// at: after `limit` polls it records HELRM_E_TIMEOUT in the error word and
// returns, exactly as a stalled stage would (self-test of the timeout path).
__global__ void k_wait_probe(long limit, int *err)
{
    pdl_begin();
    __shared__ __align__(8) u64 bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool ok = false;
    for (long it = 0; it < limit && !ok; it++) ok = mbar_try_wait(&bar, 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, (int)HELRM_E_TIMEOUT);
}

}  // namespace

namespace k {

void bsgs_tma_batch(Ctx *c, const std::vector<BsgsQuery> &qv, const u64 *const *d_keytab, const int *d_keylv,
                    const u64 *gals,
                    const u64 *const *d_diag_ptrs, const int *d_gb_index, int n_diag, int n_keys, int n1, int n2,
                    int level)
{
    const int dnum = c->dnum(level);
    HCHECK(n1 <= 64 && (n2 == 1 || n2 == 2 || n2 == 4 || n2 == 8), HELRM_E_PARAM, "BSGS tile supports n1 <= 64, n2 <= 8");
    HCHECK(dnum >= 1 && dnum <= 9 && c->N >= T, HELRM_E_PARAM, "BSGS tile supports 1..9 digits");
    TmaGals bk;
    for (int b = 0; b < 64; b++) bk.gal[b] = b < n1 ? gals[b] : 1;
    const size_t plane = (size_t)(level + 1 + c->K) * c->N;
    for (size_t q0 = 0; q0 < qv.size(); q0 += BQ) {
        const int nq = (int)std::min<size_t>(BQ, qv.size() - q0);
        TmaQueries qs = {};
        for (int q = 0; q < nq; q++) {
            qs.inner[q] = qv[q0 + q].inner;
            qs.dig[q] = qv[q0 + q].dig;
            qs.c0[q] = qv[q0 + q].c0;
            qs.c1[q] = qv[q0 + q].c1;
        }
        // per query: its keys and ciphertext once; the diagonals once per launch
        KTimer kt(c, "bsgs_fused", 8.0 * plane * nq * (2.0 * dnum * n_keys + 2.0 * n2) + 8.0 * plane * n_diag +
                                       16.0 * nq * (level + 1) * c->N);
        const u64 *const *kt_q = d_keytab + q0 * 64;
        const int *kl_q = d_keylv + q0 * 64;
#define HELRM_TMA(NN, DD) launch_tma<NN, DD>(c, qs, nq, bk, kt_q, kl_q, d_diag_ptrs, d_gb_index, n1, level)
#define HELRM_TMA_D(NN)              \
    switch (dnum) {                  \
    case 1: HELRM_TMA(NN, 1); break; \
    case 2: HELRM_TMA(NN, 2); break; \
    case 3: HELRM_TMA(NN, 3); break; \
    case 4: HELRM_TMA(NN, 4); break; \
    case 5: HELRM_TMA(NN, 5); break; \
    case 6: HELRM_TMA(NN, 6); break; \
    case 7: HELRM_TMA(NN, 7); break; \
    case 8: HELRM_TMA(NN, 8); break; \
    default: HELRM_TMA(NN, 9); break; \
    }
        switch (n2) {
        case 1: HELRM_TMA_D(1); break;
        case 2: HELRM_TMA_D(2); break;
        case 4: HELRM_TMA_D(4); break;
        default: HELRM_TMA_D(8); break;
        }
#undef HELRM_TMA_D
#undef HELRM_TMA
        c->launches++;
        CUDA_CHECK(cudaGetLastError());
    }
}

void wait_probe(Ctx *c, long limit)
{
    launch(c, k_wait_probe, 1, 32, 0, limit, c->d_err.as<int>());
    c->launches++;
    CUDA_CHECK(cudaGetLastError());
}

void bsgs_tma(Ctx *c, u64 *inner, const u64 *digits, const u64 *c0, const u64 *c1, const SwitchKey *const *keys,
              const u64 *gals, const u64 *const *d_diag_ptrs, const int *d_gb_index, int n_diag, int n1, int n2,
              int level)
{
    // the key table of this one query (pointers, then levels), staged to the device (stream ordered)
    struct {
        const u64 *ptr[64];
        int lv[64];
    } tab = {};
    int n_keys = 0;
    for (int b = 1; b < n1; b++)
        if (keys[b]) {
            tab.ptr[b] = keys[b]->data.u();
            tab.lv[b] = keys[b]->level;
            n_keys++;
        }
    DevMem d_tab(c, sizeof(tab));
    CUDA_CHECK(cudaMemcpyAsync(d_tab.ptr, &tab, sizeof(tab), cudaMemcpyHostToDevice, c->stream));
    bsgs_tma_batch(c, {{inner, digits, c0, c1}}, d_tab.as<const u64 *const>(),
                   (const int *)((const char *)d_tab.ptr + sizeof(tab.ptr)), gals, d_diag_ptrs, d_gb_index, n_diag,
                   n_keys, n1, n2, level);
}

}  // namespace k
}  // namespace helrm
