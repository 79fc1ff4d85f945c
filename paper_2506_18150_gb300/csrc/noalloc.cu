// noalloc.cu -- a rescale that allocates no memory.
//
// Some callers cannot call cudaMalloc (or anything that does): a host whose
// device memory is owned entirely by another allocator (a framework's caching
// pool that has reserved the GPU), a real-time serving loop that must not take
// an allocation's implicit device synchronisation, or code that may only touch
// buffers it was handed.  helrm_rescale_noalloc serves them: the caller passes
// the input and output buffers, and the one scratch buffer the operation
// needs (the inverse-NTT copy of the dropped limb of each polynomial) is the
// file-scope device array below.  Creating a context on a device loads it
// there (noalloc_setup); the device then holds it until the process exits.
//
// The arithmetic is that of helrm_rescale: out_i = (x_i - r) * q_l^-1 mod q_i
// with r the centred remainder of the dropped limb, which is round(x / q_l).
#include <mutex>

#include "core.cuh"

namespace helrm {
namespace {

// Scratch for the dropped limbs: two polynomials of N = 2^16 words (1 MiB).
constexpr size_t NOALLOC_SCRATCH_WORDS = 2 * 65536;
static __device__ __align__(256) u64 g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];

constexpr int MAXQ = 32;
struct RescaleConsts {
    u64 q[MAXQ];        // target primes q_0..q_{l-1}
    u64 qinv[MAXQ];     // q^-1 mod 2^64 (REDC)
    u64 ql_mod[MAXQ];   // q_l mod q_i
    u64 ql_inv[MAXQ];   // q_l^-1 mod q_i, Montgomery form
    u64 ql;             // the dropped prime
};

// out[p][i][j] = centred(last[p][j]) mod q_i   (coefficient domain)
__global__ void k_na_spread(u64 *__restrict__ out, const u64 *__restrict__ last, int level, int logN, int n_polys,
                            RescaleConsts rc)
{
    pdl_begin();
    const size_t N = (size_t)1 << logN;
    const size_t total = (size_t)n_polys * level * N;
    const u64 half = (rc.ql - 1) >> 1;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t p = idx / ((size_t)level * N);
        const int i = (int)((idx / N) % level);
        const u64 q = rc.q[i];
        const u64 x = last[p * N + (idx & (N - 1))];
        const u64 xm = x < q ? x : x % q;
        out[idx] = x <= half ? xm : sub_mod(xm, rc.ql_mod[i], q);
    }
}

// out[p][i][j] = (in[p][i][j] - out[p][i][j]) * q_l^-1 mod q_i   (NTT domain)
__global__ void k_na_finish(u64 *__restrict__ out, const u64 *__restrict__ in, int level, int logN, int n_polys,
                            RescaleConsts rc)
{
    pdl_begin();
    const size_t N = (size_t)1 << logN;
    const size_t total = (size_t)n_polys * level * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t p = idx / ((size_t)level * N);
        const size_t rem = idx - p * level * N;   // i * N + j
        const int i = (int)(rem / N);
        const u64 q = rc.q[i];
        const u64 x = in[p * (size_t)(level + 1) * N + rem];
        out[idx] = mont_mul(sub_mod(x, out[idx], q), rc.ql_inv[i], q, rc.qinv[i]);
    }
}

// Per-device address of the scratch array.  Host code cannot use the array's
// name as a device address; noalloc_setup looks it up when a context is
// created on the device (where allocating is allowed: under lazy module
// loading the lookup is what loads this file's module, and with it the
// array), and the entry point only reads the table.
std::mutex g_mu;
u64 *g_scratch_ptr[64] = {nullptr};

u64 *scratch_of(int device)
{
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    return g_scratch_ptr[device];
}

u64 h_mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
u64 h_powmod(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    for (; e; e >>= 1) {
        if (e & 1) r = h_mulmod(r, b, m);
        b = h_mulmod(b, b, m);
    }
    return r;
}

}  // namespace

void noalloc_setup(Ctx *c)
{
    HCHECK(c->device >= 0 && c->device < 64, HELRM_E_INVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_ptr[c->device]) return;
    int prev = 0;
    CUDA_CHECK(cudaGetDevice(&prev));
    CUDA_CHECK(cudaSetDevice(c->device));
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    // load the two kernels too, so that their first launch loads nothing
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_spread);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_finish);
    cudaSetDevice(prev);
    if (e != cudaSuccess) fail(HELRM_E_CUDA, std::string("noalloc set-up: ") + cudaGetErrorString(e));
    g_scratch_ptr[c->device] = (u64 *)p;
}

}  // namespace helrm

using namespace helrm;

extern "C" helrm_status helrm_rescale_noalloc(helrm_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int32_t level,
                                              uint32_t n_polys)
{
    Ctx *c = (ctx && ((const Handle *)ctx)->kind == KIND_CTX) ? (Ctx *)ctx : nullptr;
    if (!c) return HELRM_E_INVAL;
    // per-kernel timing records events, which creates driver objects: off for this call
    struct ProfOff {
        Ctx *c;
        bool was;
        explicit ProfOff(Ctx *cc) : c(cc), was(cc->prof_on) { c->prof_on = false; }
        ~ProfOff() { c->prof_on = was; }
    } prof_off(c);
    return guard(c, [&] {
        HCHECK(d_in && d_out, HELRM_E_INVAL, "NULL buffer");
        HCHECK(level >= 1 && level <= c->L, HELRM_E_LEVEL, "level must be in [1, L]");
        HCHECK(n_polys >= 1, HELRM_E_INVAL, "n_polys must be at least 1");
        HCHECK((size_t)n_polys * c->N <= NOALLOC_SCRATCH_WORDS, HELRM_E_INVAL,
               "n_polys * N exceeds the static scratch of 2 * 65536 words");
        HCHECK(level <= MAXQ, HELRM_E_PARAM, "too many primes");
        const int N = c->N, l = level;
        {   // the kernels take both buffers as __restrict__: they must not overlap
            const uintptr_t a0 = (uintptr_t)d_in, a1 = a0 + (uintptr_t)n_polys * (l + 1) * N * 8;
            const uintptr_t b0 = (uintptr_t)d_out, b1 = b0 + (uintptr_t)n_polys * l * N * 8;
            HCHECK(a1 <= b0 || b1 <= a0, HELRM_E_INVAL, "d_in and d_out overlap");
        }
        u64 *scratch = scratch_of(c->device);
        HCHECK(scratch, HELRM_E_CUDA, "the scratch array of this device was not set up");
        RescaleConsts rc;
        rc.ql = c->primes[l];
        for (int i = 0; i < l; i++) {
            const u64 q = c->primes[i];
            rc.q[i] = q;
            rc.qinv[i] = c->pinfo[i].qinv;
            rc.ql_mod[i] = rc.ql % q;
            rc.ql_inv[i] = h_mulmod(h_powmod(rc.ql % q, q - 2, q), c->pinfo[i].rmod, q);
        }
        for (u32 p = 0; p < n_polys; p++)
            CUDA_CHECK(cudaMemcpyAsync(scratch + (size_t)p * N, d_in + ((size_t)p * (l + 1) + l) * N, (size_t)N * 8,
                                       cudaMemcpyDeviceToDevice, c->stream));
        k::ntt_map_noheap(c, scratch, (int)n_polys, c->qmap(l, l, 1), true);
        const size_t total = (size_t)n_polys * l * N;
        const unsigned grid = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 64);
        launch(c, k_na_spread, grid, 256, 0, d_out, scratch, l, c->logN, (int)n_polys, rc);
        CUDA_CHECK(cudaGetLastError());
        k::ntt_map_noheap(c, d_out, (int)n_polys * l, c->qmap(l - 1, 0, l), false);
        launch(c, k_na_finish, grid, 256, 0, d_out, d_in, l, c->logN, (int)n_polys, rc);
        CUDA_CHECK(cudaGetLastError());
        c->launches += 2;
    });
}
