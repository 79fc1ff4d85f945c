// peak.cu -- the integer ceiling the NTT and the inner products are measured
// against: the register-resident rate of their arithmetic (helrm_alu_peak).
#include "butterfly.cuh"

namespace helrm {
namespace {

// Register-resident throughput of the transform's arithmetic (the integer
// ceiling the NTT is measured against).  Every thread keeps 8 residues and 7
// twiddles in registers and repeats, `iters` times, one of:
//  PEAK_CT    a forward radix-8 round: 12 lazy Cooley-Tukey butterflies
//             (bfly_ct, the code the forward passes run);
//  PEAK_GS    an inverse radix-8 round: 12 Gentleman-Sande butterflies (bfly_gs);
//  PEAK_MAC   8 carry-chained 64 x 64 -> 128-bit multiply-accumulates
//             (Acc128::mac, the key and diagonal inner products);
//  PEAK_SHOUP 8 fully reduced Shoup products (shoup_mul);
//  PEAK_MAC4  the sums of PEAK_MAC from four 32 x 32 -> 64-bit products and
//             explicit carries;
//  PEAK_MAC40 the same for operands below 2^40: three carry-free 64-bit
//             column sums of 20 x 20-bit products.
// Nothing is loaded or stored inside the loop; the result is written once so
// the work cannot be dropped.
enum PeakKind { PEAK_CT = 0, PEAK_GS = 1, PEAK_MAC = 2, PEAK_SHOUP = 3, PEAK_MAC4 = 4, PEAK_MAC40 = 5 };
template <int KIND>
__global__ void __launch_bounds__(256) k_alu_peak(u64 *__restrict__ out, const PrimeInfo *__restrict__ pinfo,
                                                  const ulonglong2 *__restrict__ tw, int pid, int logN, int iters)
{
    const u64 q = pinfo[pid].q, q2 = 2 * q;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const ulonglong2 *twp = tw + ((size_t)pid << logN);
    u64 v[8];
    ulonglong2 w[7];
#pragma unroll
    for (int j = 0; j < 7; j++) w[j] = twp[1 + ((t * 7 + j) & 255)];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = w[k % 7].x ^ (u64)(t * 8 + k);
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = v[k] >= q ? v[k] - q : v[k];
    if (KIND == PEAK_MAC) {
        Acc128 acc[8];
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int k = 0; k < 8; k++) acc[k].mac(v[k], w[k % 7].x, q);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = acc[k].lo ^ acc[k].hi;
    } else if (KIND == PEAK_MAC4) {
        // the same 128-bit sums from four 32 x 32 -> 64-bit products and
        // explicit carries
        u64 lo[8] = {0}, hi[8] = {0};
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const u64 a = v[k], b = w[k % 7].x;
                const u64 p00 = (u64)(u32)a * (u32)b, p01 = (u64)(u32)a * (u32)(b >> 32);
                const u64 p10 = (u64)(u32)(a >> 32) * (u32)b, p11 = (u64)(u32)(a >> 32) * (u32)(b >> 32);
                const u64 mid = p01 + p10;
                const u64 lo_add = p00 + (mid << 32);
                const u64 hi_add = p11 + (mid >> 32) + (mid < p01 ? (1ull << 32) : 0) + (lo_add < p00 ? 1 : 0);
                lo[k] += lo_add;
                hi[k] += hi_add + (lo[k] < lo_add ? 1 : 0);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = lo[k] ^ hi[k];
    } else if (KIND == PEAK_MAC40) {
        // operands below 2^40 as two 20-bit halves: three 64-bit column sums of
        // 40-bit products, no carries (2^24 terms fit)
        u64 c0[8] = {0}, c1[8] = {0}, c2[8] = {0};
        u32 a0[8], a1[8], b0[7], b1[7];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const u64 a = v[k] & ((1ull << 40) - 1);
            a0[k] = (u32)(a & 0xFFFFF);
            a1[k] = (u32)(a >> 20);
        }
#pragma unroll
        for (int j = 0; j < 7; j++) {
            const u64 b = w[j].x & ((1ull << 40) - 1);
            b0[j] = (u32)(b & 0xFFFFF);
            b1[j] = (u32)(b >> 20);
        }
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                c0[k] += (u64)a0[k] * b0[k % 7];
                c1[k] += (u64)a0[k] * b1[k % 7] + (u64)a1[k] * b0[k % 7];
                c2[k] += (u64)a1[k] * b1[k % 7];
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = c0[k] ^ c1[k] ^ c2[k];
    } else {
        for (int it = 0; it < iters; it++) {
            if (KIND == PEAK_CT) {
#pragma unroll
                for (int k = 0; k < 4; k++) bfly_ct(v[k], v[k + 4], w[0].x, w[0].y, q, q2);
#pragma unroll
                for (int k = 0; k < 8; k += 4) {
                    bfly_ct(v[k], v[k + 2], w[1 + k / 4].x, w[1 + k / 4].y, q, q2);
                    bfly_ct(v[k + 1], v[k + 3], w[1 + k / 4].x, w[1 + k / 4].y, q, q2);
                }
#pragma unroll
                for (int k = 0; k < 8; k += 2) bfly_ct(v[k], v[k + 1], w[3 + k / 2].x, w[3 + k / 2].y, q, q2);
            } else if (KIND == PEAK_GS) {
#pragma unroll
                for (int k = 0; k < 8; k += 2) bfly_gs(v[k], v[k + 1], w[3 + k / 2].x, w[3 + k / 2].y, q, q2);
#pragma unroll
                for (int k = 0; k < 8; k += 4) {
                    bfly_gs(v[k], v[k + 2], w[1 + k / 4].x, w[1 + k / 4].y, q, q2);
                    bfly_gs(v[k + 1], v[k + 3], w[1 + k / 4].x, w[1 + k / 4].y, q, q2);
                }
#pragma unroll
                for (int k = 0; k < 4; k++) bfly_gs(v[k], v[k + 4], w[0].x, w[0].y, q, q2);
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++) v[k] = shoup_mul(v[k], w[k % 7].x, w[k % 7].y, q);
            }
        }
    }
    u64 r = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) r ^= v[k];
    out[t] = r;
}

}  // namespace

namespace k {

double alu_peak(Ctx *c, int kind, int blocks_per_sm, int iters)
{
    HCHECK(kind >= PEAK_CT && kind <= PEAK_MAC40, HELRM_E_INVAL, "unknown peak kind");
    HCHECK(blocks_per_sm >= 1 && blocks_per_sm <= 32 && iters >= 1, HELRM_E_INVAL, "bad peak launch shape");
    const int blocks = c->n_sms * blocks_per_sm, threads = 256;
    DevMem out(c, (size_t)blocks * threads * 8);
    const int pid = c->nP() > 1 ? 1 : 0;
    const ulonglong2 *tw = c->d_tw_fwd.as<ulonglong2>();
    auto run = [&](int n) {
        void (*kern)(u64 *, const PrimeInfo *, const ulonglong2 *, int, int, int) =
            kind == PEAK_CT ? k_alu_peak<PEAK_CT> : kind == PEAK_GS ? k_alu_peak<PEAK_GS>
            : kind == PEAK_MAC ? k_alu_peak<PEAK_MAC> : kind == PEAK_SHOUP ? k_alu_peak<PEAK_SHOUP>
            : kind == PEAK_MAC4 ? k_alu_peak<PEAK_MAC4> : k_alu_peak<PEAK_MAC40>;
        kern<<<blocks, threads, 0, c->stream>>>(out.u(), c->d_pinfo.as<PrimeInfo>(), tw, pid, c->logN, n);
        CUDA_CHECK(cudaGetLastError());
    };
    run(std::max(1, iters / 8));   // warm-up (clocks, instruction cache)
    cudaEvent_t e0, e1;
    CUDA_CHECK(cudaEventCreate(&e0));
    CUDA_CHECK(cudaEventCreate(&e1));
    CUDA_CHECK(cudaEventRecord(e0, c->stream));
    run(iters);
    CUDA_CHECK(cudaEventRecord(e1, c->stream));
    CUDA_CHECK(cudaEventSynchronize(e1));
    float ms = 0;
    CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->launches += 2;
    const double per_iter = (kind == PEAK_CT || kind == PEAK_GS) ? 12.0 : 8.0;   // butterflies, else products
    return (double)blocks * threads * iters * per_iter / (ms / 1000.0);
}

}  // namespace k
}  // namespace helrm
