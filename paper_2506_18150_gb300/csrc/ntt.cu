// ntt.cu -- 64-bit negacyclic NTT / inverse NTT, batched over limbs.
//
// Forward: merged Cooley-Tukey (twiddle psi^brv(m+i) at stage m, block i),
// standard order in, bit-reversed evaluation order out:
// ahat[i] = a(psi^(2 brv(i) + 1)).  Inverse: merged Gentleman-Sande with
// psi^-brv(m+i), then 1/N.  Twiddles use Shoup's precomputed quotient.
//
// N = N1 * N2 is split into two shared-memory passes, each reading and
// writing every limb once: the first log2(N1) stages pair elements N/2..N2
// apart, so each of the N2 columns (stride N2) is an independent N1-point
// problem; the remaining log2(N2) stages stay inside contiguous rows of N2.
// A CTA holds a tile of up to 4096 words (32 KB): C columns x N1 rows for the
// column pass (C consecutive words per row keep the loads coalesced), or R
// whole rows for the row pass.  When a whole ciphertext is transformed, the
// intermediate between the two passes is L2-resident (129 MB L2).
#include "core.cuh"

namespace helrm {
namespace {

constexpr int TILE = 4096;

struct Split {
    int logN, logN1, N1, N2, C, R;
};
Split split_of(int logN)
{
    Split s;
    s.logN = logN;
    s.logN1 = logN / 2;
    s.N1 = 1 << s.logN1;
    s.N2 = 1 << (logN - s.logN1);
    s.C = std::min(TILE / s.N1, s.N2);
    s.R = std::min(TILE / s.N2, s.N1);
    return s;
}

__global__ void __launch_bounds__(512) k_fwd_cols(u64 *data, int logN, int logN1, int logC,
                                                   const ulonglong2 *__restrict__ tw_all,
                                                   const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    extern __shared__ u64 sm[];
    const int N = 1 << logN, N1 = 1 << logN1, N2 = N >> logN1, C = 1 << logC;
    const int pid = map.pid(blockIdx.y);
    const u64 q = pinfo[pid].q;
    const ulonglong2 *tw = tw_all + (size_t)pid * N;
    u64 *a = data + (size_t)blockIdx.y * N;
    const int c0 = blockIdx.x * C;
    const int tile = N1 * C;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int r = idx >> logC, c = idx & (C - 1);
        sm[idx] = a[(size_t)r * N2 + c0 + c];
    }
    __syncthreads();
    for (int s = 0; s < logN1; s++) {
        const int m = 1 << s;
        const int logt = logN1 - s - 1;
        for (int b = threadIdx.x; b < tile / 2; b += blockDim.x) {
            int c = b & (C - 1), pr = b >> logC;
            int g = pr >> logt, pos = pr & ((1 << logt) - 1);
            int r = (g << (logt + 1)) + pos;
            ulonglong2 w = tw[m + g];
            int i0 = (r << logC) + c, i1 = ((r + (1 << logt)) << logC) + c;
            u64 u = sm[i0];
            u64 v = shoup_mul(sm[i1], w.x, w.y, q);
            sm[i0] = add_mod(u, v, q);
            sm[i1] = sub_mod(u, v, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int r = idx >> logC, c = idx & (C - 1);
        a[(size_t)r * N2 + c0 + c] = sm[idx];
    }
}

__global__ void __launch_bounds__(512) k_fwd_rows(u64 *data, int logN, int logN1, int logR,
                                                   const ulonglong2 *__restrict__ tw_all,
                                                   const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    extern __shared__ u64 sm[];
    const int N = 1 << logN, logN2 = logN - logN1, N2 = 1 << logN2, R = 1 << logR;
    const int pid = map.pid(blockIdx.y);
    const u64 q = pinfo[pid].q;
    const ulonglong2 *tw = tw_all + (size_t)pid * N;
    const int r0 = blockIdx.x * R;
    u64 *a = data + (size_t)blockIdx.y * N + (size_t)r0 * N2;
    const int tile = R * N2;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) sm[idx] = a[idx];
    __syncthreads();
    for (int s = logN1; s < logN; s++) {
        const int m = 1 << s;
        const int logt = logN - s - 1;   // t = N / 2m <= N2 / 2
        for (int b = threadIdx.x; b < tile / 2; b += blockDim.x) {
            int row = b >> (logN2 - 1), x = b & ((N2 >> 1) - 1);
            int g = x >> logt, pos = x & ((1 << logt) - 1);
            int jl = (g << (logt + 1)) + pos;
            int i = ((r0 + row) << (logN2 - 1 - logt)) + g;
            ulonglong2 w = tw[m + i];
            int i0 = (row << logN2) + jl, i1 = i0 + (1 << logt);
            u64 u = sm[i0];
            u64 v = shoup_mul(sm[i1], w.x, w.y, q);
            sm[i0] = add_mod(u, v, q);
            sm[i1] = sub_mod(u, v, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) a[idx] = sm[idx];
}

__global__ void __launch_bounds__(512) k_inv_rows(u64 *data, int logN, int logN1, int logR,
                                                   const ulonglong2 *__restrict__ tw_all,
                                                   const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    extern __shared__ u64 sm[];
    const int N = 1 << logN, logN2 = logN - logN1, N2 = 1 << logN2, R = 1 << logR;
    const int pid = map.pid(blockIdx.y);
    const u64 q = pinfo[pid].q;
    const ulonglong2 *tw = tw_all + (size_t)pid * N;
    const int r0 = blockIdx.x * R;
    u64 *a = data + (size_t)blockIdx.y * N + (size_t)r0 * N2;
    const int tile = R * N2;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) sm[idx] = a[idx];
    __syncthreads();
    for (int s = logN - 1; s >= logN1; s--) {
        const int m = 1 << s;
        const int logt = logN - s - 1;
        for (int b = threadIdx.x; b < tile / 2; b += blockDim.x) {
            int row = b >> (logN2 - 1), x = b & ((N2 >> 1) - 1);
            int g = x >> logt, pos = x & ((1 << logt) - 1);
            int jl = (g << (logt + 1)) + pos;
            int i = ((r0 + row) << (logN2 - 1 - logt)) + g;
            ulonglong2 w = tw[m + i];
            int i0 = (row << logN2) + jl, i1 = i0 + (1 << logt);
            u64 u = sm[i0], v = sm[i1];
            sm[i0] = add_mod(u, v, q);
            sm[i1] = shoup_mul(sub_mod(u, v, q), w.x, w.y, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) a[idx] = sm[idx];
}

__global__ void __launch_bounds__(512) k_inv_cols(u64 *data, int logN, int logN1, int logC,
                                                   const ulonglong2 *__restrict__ tw_all,
                                                   const ulonglong2 *__restrict__ ninv,
                                                   const PrimeInfo *__restrict__ pinfo, LimbMap map)
{
    extern __shared__ u64 sm[];
    const int N = 1 << logN, N1 = 1 << logN1, N2 = N >> logN1, C = 1 << logC;
    const int pid = map.pid(blockIdx.y);
    const u64 q = pinfo[pid].q;
    const ulonglong2 *tw = tw_all + (size_t)pid * N;
    const ulonglong2 ni = ninv[pid];
    u64 *a = data + (size_t)blockIdx.y * N;
    const int c0 = blockIdx.x * C;
    const int tile = N1 * C;
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int r = idx >> logC, c = idx & (C - 1);
        sm[idx] = a[(size_t)r * N2 + c0 + c];
    }
    __syncthreads();
    for (int s = logN1 - 1; s >= 0; s--) {
        const int m = 1 << s;
        const int logt = logN1 - s - 1;
        for (int b = threadIdx.x; b < tile / 2; b += blockDim.x) {
            int c = b & (C - 1), pr = b >> logC;
            int g = pr >> logt, pos = pr & ((1 << logt) - 1);
            int r = (g << (logt + 1)) + pos;
            ulonglong2 w = tw[m + g];
            int i0 = (r << logC) + c, i1 = ((r + (1 << logt)) << logC) + c;
            u64 u = sm[i0], v = sm[i1];
            sm[i0] = add_mod(u, v, q);
            sm[i1] = shoup_mul(sub_mod(u, v, q), w.x, w.y, q);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < tile; idx += blockDim.x) {
        int r = idx >> logC, c = idx & (C - 1);
        a[(size_t)r * N2 + c0 + c] = shoup_mul(sm[idx], ni.x, ni.y, q);
    }
}

int ilog2(int x)
{
    int r = 0;
    while ((1 << r) < x) r++;
    return r;
}

}  // namespace

namespace k {

void ntt_fwd(Ctx *c, u64 *data, int n_limbs, LimbMap map)
{
    if (n_limbs <= 0) return;
    Split s = split_of(c->logN);
    int tc = s.N1 * s.C, tr = s.R * s.N2;
    dim3 gc(s.N2 / s.C, n_limbs), gr(s.N1 / s.R, n_limbs);
    k_fwd_cols<<<gc, std::min(512, tc / 2), tc * 8, c->stream>>>(
        data, s.logN, s.logN1, ilog2(s.C), c->d_tw_fwd.as<ulonglong2>(), c->d_pinfo.as<PrimeInfo>(), map);
    k_fwd_rows<<<gr, std::min(512, tr / 2), tr * 8, c->stream>>>(
        data, s.logN, s.logN1, ilog2(s.R), c->d_tw_fwd.as<ulonglong2>(), c->d_pinfo.as<PrimeInfo>(), map);
    c->launches += 2;
    CUDA_CHECK(cudaGetLastError());
}

void ntt_inv(Ctx *c, u64 *data, int n_limbs, LimbMap map)
{
    if (n_limbs <= 0) return;
    Split s = split_of(c->logN);
    int tc = s.N1 * s.C, tr = s.R * s.N2;
    dim3 gc(s.N2 / s.C, n_limbs), gr(s.N1 / s.R, n_limbs);
    k_inv_rows<<<gr, std::min(512, tr / 2), tr * 8, c->stream>>>(
        data, s.logN, s.logN1, ilog2(s.R), c->d_tw_inv.as<ulonglong2>(), c->d_pinfo.as<PrimeInfo>(), map);
    k_inv_cols<<<gc, std::min(512, tc / 2), tc * 8, c->stream>>>(
        data, s.logN, s.logN1, ilog2(s.C), c->d_tw_inv.as<ulonglong2>(), c->d_ninv.as<ulonglong2>(),
        c->d_pinfo.as<PrimeInfo>(), map);
    c->launches += 2;
    CUDA_CHECK(cudaGetLastError());
}

}  // namespace k
}  // namespace helrm
