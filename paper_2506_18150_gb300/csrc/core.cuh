// core.cuh -- internal declarations of the GB300 HE-LRM library.
//
// Device words are u64 residues in [0, q).  Two multiplication forms are used:
//  * Montgomery (R = 2^64): constant operands (keys, diagonals, masks, base
//    conversion factors) are stored as b*R mod q, so REDC(a * bR) = a*b mod q
//    in one reduction; a 128-bit sum of such products is reduced once.
//  * Shoup: NTT twiddles carry w' = floor(w 2^64 / q), so a*w mod q costs one
//    high and two low 64-bit products.
// GB300 has no 64x64 multiplier: each 64-bit product is a short IMAD
// sequence, which is why the constant-operand forms matter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/helrm.h"

namespace helrm {

using u64 = uint64_t;
using u32 = uint32_t;
using i64 = int64_t;
using u128 = unsigned __int128;

// ----------------------------------------------------------------- errors
struct Error {
    helrm_status code;
    std::string msg;
};
[[noreturn]] void fail(helrm_status code, const std::string &msg);
#define HCHECK(cond, code, msg)                 \
    do {                                        \
        if (!(cond)) ::helrm::fail((code), (msg)); \
    } while (0)
#define CUDA_CHECK(x)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess)                                                              \
            ::helrm::fail(HELRM_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));   \
    } while (0)

// ----------------------------------------------------------- modular math
struct PrimeInfo {
    u64 q;      // the prime
    u64 qinv;   // q^-1 mod 2^64
    u64 r2;     // 2^128 mod q (to enter Montgomery form)
    u64 rmod;   // 2^64 mod q
};

__host__ __device__ __forceinline__ u64 mulhi64(u64 a, u64 b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((u128)a * b) >> 64);
#endif
}

// (hi 2^64 + lo) 2^-64 mod q, for hi < q.  m q has low word lo, so the
// difference is an exact multiple of 2^64: result = hi - mulhi(m, q), in (-q, q).
__host__ __device__ __forceinline__ u64 redc(u64 hi, u64 lo, u64 q, u64 qinv)
{
    u64 m = lo * qinv;
    u64 mh = mulhi64(m, q);
    u64 r = hi - mh;
    return hi < mh ? r + q : r;
}
// a * b mod q with b in Montgomery form (b R mod q, b < q); any a < 2^64.
__host__ __device__ __forceinline__ u64 mont_mul(u64 a, u64 b_mont, u64 q, u64 qinv)
{
    return redc(mulhi64(a, b_mont), a * b_mont, q, qinv);
}
// a * b mod q for two plain residues: two reductions (a b R^-1, then * R^2 R^-1).
__host__ __device__ __forceinline__ u64 mul_mod(u64 a, u64 b, u64 q, u64 qinv, u64 r2)
{
    return mont_mul(mont_mul(a, b, q, qinv), r2, q, qinv);
}
__host__ __device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q)
{
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__host__ __device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q)
{
    return a >= b ? a - b : a + q - b;
}
// Shoup: a * w mod q with wp = floor(w 2^64 / q), w < q, any a < 2^64.
__host__ __device__ __forceinline__ u64 shoup_mul(u64 a, u64 w, u64 wp, u64 q)
{
    u64 qh = mulhi64(a, wp);
    u64 r = a * w - qh * q;
    return r >= q ? r - q : r;
}
// 128-bit sum of products, reduced once at the end.  Every prime is below
// 2^60, so a product of two residues is below 2^120 and up to 256 of them add
// up without overflowing 128 bits: the terms are accumulated with a carry
// chain and no reduction in between.  The result is sum * 2^-64 mod q (REDC),
// which needs the high word below q.  reduce(): at most 16 terms, each a
// product of a value below 2^60 and a residue mod q, so hi < 16 * 2^60 * q /
// 2^64 = q already (every inner product of a key switch or a base
// conversion).  reduce_long(): up to 256 terms; the high word is first
// brought below q by a Montgomery product with R mod q (multiples of q 2^64
// do not change the value mod q).
struct Acc128 {
    u64 lo = 0, hi = 0;
    __host__ __device__ __forceinline__ void mac(u64 a, u64 b, u64 /*q*/)
    {
#ifdef __CUDA_ARCH__
        asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
            "madc.hi.u64 %1, %2, %3, %1;"
            : "+l"(lo), "+l"(hi)
            : "l"(a), "l"(b));
#else
        const u128 s = ((u128)hi << 64 | lo) + (u128)a * b;
        lo = (u64)s;
        hi = (u64)(s >> 64);
#endif
    }
    __host__ __device__ __forceinline__ u64 reduce(u64 q, u64 qinv) const { return redc(hi, lo, q, qinv); }
    __host__ __device__ __forceinline__ u64 reduce_long(u64 q, u64 qinv, u64 one_mont) const
    {
        return redc(mont_mul(hi, one_mont, q, qinv), lo, q, qinv);
    }
};

// Limb l of a level-ell QP polynomial uses prime q_l for l <= ell, else p_{l-ell-1}
// (global prime index L+1+(l-ell-1)).  `off` shifts the first limb; a non-zero
// `period` restarts the numbering every `period` limbs (several polynomials of
// the same basis stored back to back, e.g. both halves of a ciphertext).
struct LimbMap {
    int off;         // index of this array's first limb in the level's QP numbering
    int qc;          // number of Q limbs in the level's basis (ell + 1)
    int pbase;       // global prime index of p_0 (L + 1)
    int period = 0;  // 0 = no repetition
    __host__ __device__ __forceinline__ int pid(int l) const
    {
        int x = (period ? l % period : l) + off;
        return x < qc ? x : pbase + (x - qc);
    }
};

// ----------------------------------------------------------------- context
struct Ctx;

// Device buffer owned by a handle; freed stream-ordered on the context's stream.
struct DevMem {
    Ctx *ctx = nullptr;
    void *ptr = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(Ctx *c, size_t b);
    ~DevMem();
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    DevMem(DevMem &&o) noexcept { *this = std::move(o); }
    DevMem &operator=(DevMem &&o) noexcept;
    u64 *u() const { return (u64 *)ptr; }
    template <class T>
    T *as() const { return (T *)ptr; }
};

enum Kind : u32 {
    KIND_CTX = 0x48E10001u,
    KIND_SK,
    KIND_EVK,
    KIND_PT,
    KIND_CT,
    KIND_PTMAT,
    KIND_EMB,
    KIND_MODEL,
    KIND_BATCH,
    KIND_SERVER,
    KIND_BOOT,
};

struct Handle {
    u32 kind;
    explicit Handle(u32 k) : kind(k) {}
    virtual ~Handle() { kind = 0; }
};

// Device tables for one fast base conversion (src primes -> dst primes).
struct BConvTable {
    int n_src = 0, n_dst = 0;
    DevMem tab;      // layout: context.cu, make_bconv
    DevMem iscale;   // ulonglong2 [n_src]: N^-1 [(Q/q_s)^-1]_{q_s} and its Shoup quotient
    // the Montgomery constants [Q/q_s]_{p_k} of destination k, stride n_dst
    const u64 *hcol(int k) const { return tab.u() + 2 + 4 * n_src + 3 * n_dst + k; }
    const ulonglong2 *scale(int s) const { return iscale.as<ulonglong2>() + s; }
};

struct Ctx : Handle {
    int device = 0;
    int n_sms = 152;           // streaming multiprocessors of the device
    cudaStream_t stream = nullptr;
    int logN = 0, N = 0, n_slots = 0, L = 0, K = 0, alpha = 1;
    double delta = 0;
    std::vector<u64> primes;   // q_0..q_L, p_0..p_{K-1}
    std::vector<u64> psi;      // primitive 2N-th roots
    std::vector<PrimeInfo> pinfo;
    DevMem d_pinfo;            // PrimeInfo[nP]
    DevMem d_tw_fwd;           // ulonglong2 [nP][N]: psi^brv(k), Shoup
    DevMem d_tw_inv;           // ulonglong2 [nP][N]: psi^-brv(k), Shoup
    DevMem d_ninv;             // ulonglong2 [nP]: N^-1, Shoup
    DevMem d_fft_tw;           // double2 [N/2]: e^(-2 pi i t / N)
    DevMem d_slot_of;          // int [N]: u -> slot j with 5^j = +-(2u+1) mod 2N
    DevMem d_u_of_slot;        // int [n]: j -> (5^j mod 2N - 1)/2
    DevMem d_pmod_mont;        // u64 [nP]: (P mod q_i) R mod q_i for i <= L, 0 for the P primes
    DevMem d_pinv_mont;        // u64 [nP]: (P^-1 mod q_i) R mod q_i for i <= L
    DevMem d_one_mont;         // u64 [nP]: R mod q_i (the constant 1 in Montgomery form)
    DevMem d_err;              // int: set by kernels that detect bad data (encoder overflow)
    std::map<std::pair<int, int>, BConvTable> modup_tab;   // (level, digit)
    std::map<int, BConvTable> moddown_tab;                 // level
    std::map<int, DevMem> rescale_tab;                     // level -> constants
    std::map<int, DevMem> mdrs_tab;                        // level -> merged ModDown + rescale constants
    u64 mem_in_use = 0, mem_cap = 0, mem_peak = 0;   // bytes held, cap, high-water mark
    // NTT launch shape per limb-count bucket (<= 4, <= 16, <= 64, more limbs per
    // launch): words per CTA tile and the CTA count (in multiples of the SM count)
    // below which tiles are split; chosen by ntt_autotune at creation
    struct NttTune {
        int tile = 1024;
        int mult = 2;
        int ept = 8;     // elements per thread (4: N = 2^16 instances only)
    };
    NttTune ntt_tune[4];
    u64 launches = 0;
    std::string last_error;
    cudaMemPool_t pool = nullptr;
    // Second streams for independent branches of one inference (Fork below):
    // one per home stream (a serving slot is a home stream), each with its own
    // memory pool, so that a block freed on the home stream is never handed
    // to the branch with a wait on the home stream inserted by the allocator.
    struct Side {
        cudaStream_t stream = nullptr;
        cudaMemPool_t pool = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
    };
    std::map<cudaStream_t, Side> sides;
    cudaMemPool_t alloc_pool = nullptr;   // set inside a branch: Ctx::alloc draws from it
    bool capturing = false;               // a graph capture is open on `stream`
    Side &side_of(cudaStream_t home);
    // optional per-kernel timing with CUDA events on the context stream
    struct ProfRec {
        const char *name;
        cudaEvent_t start, stop;
        double bytes;
    };
    bool prof_on = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t take_event();

    Ctx() : Handle(KIND_CTX) {}
    ~Ctx() override;
    int nP() const { return L + 1 + K; }
    int dnum(int level) const { return (level + 1 + alpha - 1) / alpha; }
    int digit_lo(int j) const { return j * alpha; }
    int digit_hi(int j, int level) const { return std::min((j + 1) * alpha, level + 1); }
    // level-ell QP numbering starting at limb `off`, repeating every `period` limbs
    LimbMap qmap(int level, int off = 0, int period = 0) const { return LimbMap{off, level + 1, L + 1, period}; }
    void *alloc(size_t bytes);
    void release(void *p, size_t bytes);
    u64 galois(int step) const;
    const BConvTable &modup_table(int level, int digit);
    const BConvTable &moddown_table(int level);
    const u64 *rescale_table(int level);
    const u64 *moddown_rescale_table(int level);
    // synchronise; if a kernel flagged bad data since the last check, clear and raise
    void check_device_errors();
};

// Runs f, turning every exception into a status (and the context's last
// error message); after a CUDA or out-of-memory error the runtime's pending
// error is cleared so that the next call does not report it again.  Every
// entry point of the ABI is wrapped in it.
template <class F>
helrm_status guard(Ctx *ctx, F &&f)
{
    try {
        f();
        return HELRM_OK;
    } catch (const Error &e) {
        if (ctx) ctx->last_error = e.msg;
        if (e.code == HELRM_E_CUDA || e.code == HELRM_E_NOMEM) cudaGetLastError();
        return e.code;
    } catch (const std::bad_alloc &) {
        if (ctx) ctx->last_error = "host allocation failed";
        return HELRM_E_NOMEM;
    } catch (const std::exception &e) {
        if (ctx) ctx->last_error = e.what();
        return HELRM_E_INVAL;
    } catch (...) {
        if (ctx) ctx->last_error = "unknown error";
        return HELRM_E_INVAL;
    }
}

// The allocation-free rescale's set-up for the context's device (noalloc.cu):
// looks up the device address of its static scratch array and loads its
// kernels, so that the call itself never loads a module.  Called once per
// context at creation.
void noalloc_setup(Ctx *c);

// Fork / join of an independent branch of work.  The constructor records a
// fork point on the context's stream; run(f) enqueues f's work on the side
// stream of that stream (after the fork point, allocating from the side
// pool), then restores the context's stream; join() (or the destructor)
// makes the context's stream wait for everything the branch enqueued.  Work
// enqueued on the context's stream between run() and join() overlaps the
// branch.  Inside a graph capture the same calls record a forked graph.  With
// per-kernel timing on (Ctx::prof_on) the branch runs inline instead.
class Fork {
  public:
    explicit Fork(Ctx *c);
    template <class F>
    void run(F &&f)
    {
        enter();
        try {
            f();
        } catch (...) {
            leave();
            throw;
        }
        leave();
    }
    void join();
    ~Fork();
    Fork(const Fork &) = delete;
    Fork &operator=(const Fork &) = delete;

  private:
    void enter();
    void leave();
    Ctx *c;
    cudaStream_t home;
    Ctx::Side *side;   // null: inline
    bool joined = false;
};

// Scope timer: when profiling is on, brackets the enclosed launches with a
// pair of events and the kernel's algorithmic bytes (reads + writes once).
// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_begin(): griddepcontrol.wait blocks until the grids it depends on have
// completed and their writes are visible, then launch_dependents lets the next
// grid in the stream be scheduled while this one runs, so consecutive kernels
// no longer pay a full launch latency each.  Both instructions are no-ops in
// a grid launched without the attribute.  Before pdl_begin() a kernel reads
// only tables that no kernel writes (the NTT reads its twiddles and prime
// constants there), which is what makes the early launch safe.
__device__ __forceinline__ void pdl_begin()
{
#ifdef __CUDA_ARCH__
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
// Launch on the context's stream with programmatic stream serialisation.
template <typename... KArgs, typename... Args>
void launch(Ctx *c, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

struct KTimer {
    Ctx *c;
    size_t idx = (size_t)-1;
    KTimer(Ctx *ctx, const char *name, double bytes) : c(ctx)
    {
        if (!c->prof_on) return;
        Ctx::ProfRec r{name, c->take_event(), c->take_event(), bytes};
        cudaEventRecord(r.start, c->stream);
        c->prof.push_back(r);
        idx = c->prof.size() - 1;
    }
    ~KTimer()
    {
        if (idx != (size_t)-1) cudaEventRecord(c->prof[idx].stop, c->stream);
    }
};

// ---------------------------------------------------------------- objects
struct Poly {  // (n_limbs x N) u64 in the NTT domain
    DevMem mem;
    int limbs = 0;
};

struct SecretKey : Handle {
    Ctx *ctx;
    DevMem s_ntt;    // [L+1+K][N] s in NTT form, plain residues
    DevMem s_mont;   // same in Montgomery form
    SecretKey(Ctx *c) : Handle(KIND_SK), ctx(c) {}
};

// A switching key generated up to level kl: digits j < dnum(kl), each (b_j, a_j)
// over the limbs q_0..q_kl, p_0..p_{K-1}, NTT + Montgomery form.  It serves any
// key switch at a level <= kl; a key at kl = L is the full key, and a key at a
// lower level is exactly the full key's restriction (same values).
struct SwitchKey {
    DevMem data;            // [dnum][2][kl+1+K][N]
    int dnum = 0;
    int level = 0;          // kl
};
// limb of prime pid (a Q prime <= kl or a P prime, global numbering) inside a key of level kl
__host__ __device__ __forceinline__ int key_limb(int pid, int kl, int L) { return pid <= kl ? pid : pid - L + kl; }

struct EvalKey : Handle {
    Ctx *ctx;
    u64 seed = 0;
    DevMem pk;              // [2][L+1][N] (b, a) NTT, Montgomery form
    std::unique_ptr<SwitchKey> relin;
    std::map<u64, std::unique_ptr<SwitchKey>> rot;   // galois element -> key
    EvalKey(Ctx *c) : Handle(KIND_EVK), ctx(c) {}
};

enum PtForm { PT_PLAIN = 0, PT_MONT = 1 };

struct Plaintext : Handle {
    Ctx *ctx;
    int level = 0;
    bool qp = false;        // limbs q_0..q_level (+ p_0..p_{K-1} if qp)
    int form = PT_PLAIN;
    double scale = 1;
    DevMem data;            // [limbs][N] NTT domain
    Plaintext(Ctx *c) : Handle(KIND_PT), ctx(c) {}
    int limbs() const { return level + 1 + (qp ? ctx->K : 0); }
};

struct Ciphertext : Handle {
    Ctx *ctx;
    int level = 0;
    double scale = 1;
    DevMem data;            // [2][level+1][N] NTT domain
    Ciphertext(Ctx *c) : Handle(KIND_CT), ctx(c) {}
    u64 *c0() const { return data.u(); }
    u64 *c1() const { return data.u() + (size_t)(level + 1) * ctx->N; }
};

// ----------------------------------------------------------- kernel API
// (kernels.cu / ntt.cu; all launched on ctx->stream, all counted)
namespace k {
void ntt_fwd(Ctx *c, u64 *data, int n_limbs, LimbMap map);
void ntt_inv(Ctx *c, u64 *data, int n_limbs, LimbMap map);
// One limb of a batched transform: the first pass reads src and writes dst,
// the second works on dst.  With a forward transform and ea != nullptr, the
// result is not stored in dst but as eo[i] = (ea[i] - NTT(y)[i]) * ep_scal[pid]
// (+ eb[i] when eb != nullptr; eb may equal eo).
//
// Fused fast base conversion (Sec. 2.1's ModUp / ModDown): an inverse
// transform may end with a scale of its own (scal: a Shoup pair replacing
// N^-1, e.g. N^-1 [(Q/q_s)^-1]_{q_s}), and a forward transform may compute its
// input on load as src[i] = sum_{s < fbc_n} src[s N + i] * fbc_h[s fbc_hs] mod
// q (fbc_h in Montgomery form: the column of the conversion matrix for this
// limb's prime), so the converted limbs are never written to memory.
struct NttLimb {
    const u64 *src;
    u64 *dst;
    int pid;
    const u64 *ea;
    u64 *eo;
    const u64 *eb;
    const ulonglong2 *scal = nullptr;   // inverse: replaces N^-1 (device pointer; null: N^-1)
    int fbc_n = 0;                      // forward: source limbs of the conversion (0: plain input)
    const u64 *fbc_h = nullptr;         // forward: the conversion constants (device pointer)
    int fbc_hs = 0;                     // their stride
    const u64 *rs_u = nullptr;          // merged rescale (ntt_run_rescale): top limb of u, coefficients
    const u64 *rs_add = nullptr;        //   top limb of the addend, coefficients (null: none)
};
// A ModDown merged with the rescale that follows it (forward transform of the
// Q-limbs below the dropped prime q_l): the input of limb i is
// FBC_i + P r, where r is the centred coefficient of the ModDown result's top
// limb, x = (u_l - FBC_l) P^-1 (+ add_l) mod q_l, recomputed on load from the
// same sources; the epilogue is eo = (u_i - NTT) (P q_l)^-1 + add_i q_l^-1.
// Every step is exact modular arithmetic, so the residues equal those of a
// ModDown followed by a rescale.
struct NttRescale {
    const u64 *hl;          // conversion constants of q_l (device), stride hls
    int hls, lp;            // ... and the prime id of q_l
    const u64 *pmod;        // [pid]: P R mod q
    const u64 *qlmod;       // [pid]: q_l mod q
    const u64 *pinv;        // [pid]: P^-1 R mod q
    const u64 *ep_scal;     // [pid]: (P q_l)^-1 R mod q, then at add_off + pid: q_l^-1 R mod q
    int add_off;
};
void ntt_run_rescale(Ctx *c, const std::vector<NttLimb> &limbs, const NttRescale &rs);
void ntt_run(Ctx *c, const std::vector<NttLimb> &limbs, bool inverse, const u64 *ep_scal);
// same as ntt_fwd / ntt_inv, with the launch list built on the stack (no heap use)
void ntt_map_noheap(Ctx *c, u64 *data, int n_limbs, LimbMap map, bool inverse);
// time every candidate NTT launch shape per limb-count bucket on scratch limbs
// and keep the fastest (ntt.cu); the arithmetic is the same for every shape
void ntt_autotune(Ctx *c);
// register-resident throughput of the NTT's and the inner products' arithmetic
// (kind 0: forward butterflies, 1: inverse butterflies, 2: 128-bit
// multiply-accumulates, 3: Shoup products), in operations per second
double alu_peak(Ctx *c, int kind, int blocks_per_sm, int iters);
// transform an arbitrary list of limbs (offset in limbs from base, prime id) in one launch pair
void ntt_list(Ctx *c, u64 *base, const std::vector<std::pair<u32, int>> &limbs, bool inverse);
void copy(Ctx *c, u64 *dst, const u64 *src, size_t n_words);
void zero(Ctx *c, u64 *dst, size_t n_words);
void add(Ctx *c, u64 *out, const u64 *a, const u64 *b, int n_limbs, LimbMap map);
void sub(Ctx *c, u64 *out, const u64 *a, const u64 *b, int n_limbs, LimbMap map);
void neg(Ctx *c, u64 *out, const u64 *a, int n_limbs, LimbMap map);
// out = a * b_mont (b in Montgomery form)
void mul_mont(Ctx *c, u64 *out, const u64 *a, const u64 *b_mont, int n_limbs, LimbMap map);
// out = a * b (both plain)
void mul_plain(Ctx *c, u64 *out, const u64 *a, const u64 *b, int n_limbs, LimbMap map);
// out = a * R mod q (enter Montgomery form)
void to_mont(Ctx *c, u64 *out, const u64 *a, int n_limbs, LimbMap map);
// out = a R^-1 mod q (leave Montgomery form)
void from_mont(Ctx *c, u64 *out, const u64 *a, int n_limbs, LimbMap map);
// (d0, d1, d2) (+)= (a0 b0, a0 b1 + a1 b0, a1 b1) over n_limbs limbs
void tensor(Ctx *c, u64 *d, const u64 *a0, const u64 *a1, const u64 *b0, const u64 *b1, int n_limbs, LimbMap map,
            bool accumulate);
// out_l = a_l * scal_mont[pid(l)] (one constant per limb, Montgomery form, indexed by prime)
void mul_scalar_mont(Ctx *c, u64 *out, const u64 *a, const u64 *d_scal_by_prime, int n_limbs,
                     LimbMap map);
// out = (a - b) * scal[pid]
// out = a + d_scal_by_prime[pid] (plain residues) on every coefficient of n_limbs limbs
void add_scalar(Ctx *c, u64 *out, const u64 *a, const u64 *d_scal_by_prime, int n_limbs, LimbMap map);
void sub_mul_scalar(Ctx *c, u64 *out, const u64 *a, const u64 *b, const u64 *d_scal_by_prime,
                    int n_limbs, LimbMap map);
// centred integers (int64 N) -> residues for n_limbs limbs
// n_polys polynomials (in: [n_polys][N], out: [n_polys][n_limbs][N]) in one launch
void from_signed(Ctx *c, u64 *out, const i64 *in, int n_limbs, LimbMap map, int n_polys = 1);
// an encryption's v (ternary), e0, e1 (CBD(21)) into out3[3][N], one launch
void sample_enc_noise(Ctx *c, i64 *out3, u64 seed, u32 pv, u32 pe0, u32 pe1);
// c0 = v pk0 + e0 + m, c1 = v pk1 + e1 over n_limbs limbs, one launch
void enc_combine(Ctx *c, u64 *c0, u64 *c1, const u64 *v, const u64 *e0, const u64 *e1, const u64 *m, const u64 *pk0,
                 const u64 *pk1, int n_limbs, LimbMap map);
// d_out[l][i] = sum_j dig_j[l][perm(i)] * key_j(l)[i] for the level-ell QP basis, both
// polys of the key; if c0 != null, out0 on Q limbs += P * c0[perm(i)]
// bq (optional): a QP polynomial whose image phi(bq) is added to the first
// output; accumulate: add the result to what out already holds.
void ks_inner_auto(Ctx *c, u64 *out, const u64 *digits, int dnum, const SwitchKey *key, int level,
                   u64 galois, const u64 *c0, const u64 *d_pmod_mont, const u64 *bq = nullptr,
                   bool accumulate = false);
// inner[g][2][limbs][N] = sum_b diag[(g,b)] * baby[b]
void bsgs_mac(Ctx *c, u64 *inner, const u64 *baby, int n_baby, const u64 *const *d_diag_ptrs,
              const int *d_gb_index, int n2, int n1, int limbs, LimbMap map);
void automorphism(Ctx *c, u64 *out, const u64 *in, int n_limbs, u64 galois);
// hoisted baby steps fused into the BSGS MAC (n1 <= 64, n2 in {1,2,4,8}), fed by a
// 3-stage pipeline of bulk asynchronous copies (bsgs_tma.cu); keys[b] / gals[b] for
// b < n1 (keys[0] unused); writes inner[g][2][level+1+K][N] for giant steps with diagonals
void bsgs_tma(Ctx *c, u64 *inner, const u64 *digits, const u64 *c0, const u64 *c1, const SwitchKey *const *keys,
              const u64 *gals, const u64 *const *d_diag_ptrs, const int *d_gb_index, int n_diag, int n1, int n2,
              int level);
// the same for a batch of queries of one matrix (one launch per 64 queries):
// query q reads its keys from d_keytab[q][0..63] (device, baby step b >= 1), whose
// levels are d_keylv[q][0..63]
struct BsgsQuery {
    u64 *inner;
    const u64 *dig;
    const u64 *c0;
    const u64 *c1;
};
void bsgs_tma_batch(Ctx *c, const std::vector<BsgsQuery> &qs, const u64 *const *d_keytab, const int *d_keylv,
                    const u64 *gals,
                    const u64 *const *d_diag_ptrs, const int *d_gb_index, int n_diag, int n_keys, int n1, int n2,
                    int level);
// one CTA waits (at most `limit` polls) on an mbarrier nothing arrives at, then
// records HELRM_E_TIMEOUT in the context's error word
void wait_probe(Ctx *c, long limit);
// rescale helper: coefficient-form last limb -> centred residues for ell limbs
void rescale_spread(Ctx *c, u64 *out, const u64 *last_coef, int level, int n_polys = 1);
// random
void chacha_words(Ctx *c, u32 *out, u64 seed, u32 purpose, u64 index, u64 first_word, u64 n_words);
void sample_uniform(Ctx *c, u64 *out, u64 seed, u32 purpose, u64 index, int n_limbs,
                    const int *d_limb_pid, const int *d_limb_gid);
void sample_ternary(Ctx *c, i64 *out, u64 seed, u32 purpose, u64 index);
void sample_cbd21(Ctx *c, i64 *out, u64 seed, u32 purpose, u64 index);
// exactly h coefficients in {-1, +1} at the h smallest (priority, position) pairs (one CTA)
void sample_sparse_ternary(Ctx *c, i64 *out, u64 seed, u32 purpose, int h);
// ModRaise: n_polys level-0 polynomials (limb 0, coefficient domain, in_stride words
// apart) centred mod q_0 and written as residues of n_limbs limbs ([n_polys][n_limbs][N])
void mod_raise(Ctx *c, u64 *out, const u64 *in0_coef, size_t in_stride, int n_polys, int n_limbs, LimbMap map);
// FFT encode / decode
// (d_slots_im != null: complex slots, real parts d_slots)
void encode_slots(Ctx *c, u64 *out_residues, const double *d_slots, int n_valid, int period,
                  double scale, int n_limbs, LimbMap map, i64 *d_coeffs_out, const double *d_slots_im = nullptr);
void decode_limb0(Ctx *c, double *d_slots_out, const u64 *m_coef_limb0, double scale, int n_slots);
void check_range(Ctx *c, const u64 *data, int n_limbs, LimbMap map, int *d_flag);
// selector one-hots of one query: d_tab [T][3] = (rows, offset, digits)
void pack_selector(Ctx *c, double *sel, const u64 *d_idx, const int *d_tab, int T, int base, int in_pad);
void sigmoid(Ctx *c, double *d_p, const double *d_x, int n);
}  // namespace k

// ------------------------------------------------------ scheme (scheme.cu)
Ciphertext *new_ct(Ctx *c, int level, double scale);
void ks_modup(Ctx *c, const u64 *poly_ntt, int level, u64 *digits_out);
// the launch lists of a ModUp / one half of a ModDown with the base conversion
// fused into the transforms (appended to inv and fwd; coef: (level+1) limbs of
// scratch; pc: K limbs, y: level+1 limbs of scratch)
void modup_limbs(Ctx *c, int level, const u64 *poly, u64 *coef, u64 *digits, std::vector<k::NttLimb> &inv,
                 std::vector<k::NttLimb> &fwd);
void moddown_limbs(Ctx *c, int level, const u64 *qp, u64 *pc, u64 *y, u64 *out, const u64 *add,
                   std::vector<k::NttLimb> &inv, std::vector<k::NttLimb> &fwd);
void ks_moddown(Ctx *c, const u64 *qp_ntt, int level, u64 *out_ntt);
// out_h = ModDown(u_h) (+ add_h when add_h != nullptr; add_h may equal out_h)
void ks_moddown2(Ctx *c, const u64 *u, int level, u64 *out0, u64 *out1, const u64 *add0 = nullptr,
                 const u64 *add1 = nullptr);
Ciphertext *ct_rescale(Ctx *c, const Ciphertext *a);
Ciphertext *ct_add(Ctx *c, const Ciphertext *a, const Ciphertext *b, bool subtract = false);
Ciphertext *ct_add_pt(Ctx *c, const Ciphertext *a, const Plaintext *pt);
Ciphertext *ct_mul_pt(Ctx *c, const Ciphertext *a, const Plaintext *pt);
Ciphertext *ct_drop(Ctx *c, const Ciphertext *a, int level);
void ct_rotate_hoisted(Ctx *c, const EvalKey *evk, const Ciphertext *a, const std::vector<int> &steps,
                       std::vector<Ciphertext *> &outs);
Ciphertext *ct_rotate(Ctx *c, const EvalKey *evk, const Ciphertext *a, int step);
// X -> X^g and the key switch back to s (g = 2N - 1: complex conjugation of every slot)
Ciphertext *ct_apply_galois(Ctx *c, const EvalKey *evk, const Ciphertext *a, u64 g);
void ct_tensor_acc(Ctx *c, u64 *d012, const Ciphertext *a, const Ciphertext *b, bool accumulate);
Ciphertext *ct_relin(Ctx *c, const EvalKey *evk, const u64 *d012, int level, double scale);
Ciphertext *ct_mul(Ctx *c, const EvalKey *evk, const Ciphertext *a, const Ciphertext *b);
// h_slots_im != null: complex slots (h_slots the real parts)
Plaintext *pt_encode(Ctx *c, const double *h_slots, int n_slots, int period, int level, bool qp,
                     double scale, int form, const double *h_slots_im = nullptr);
Plaintext *pt_encode_dev(Ctx *c, const double *d_slots, int n_valid, int period, int level, double scale);
Plaintext *pt_from_signed(Ctx *c, const i64 *h_coeffs, int level, bool qp, double scale, int form);
void pt_export_signed(Ctx *c, const Plaintext *pt, i64 *h_out);
// h = 0: dense ternary CBD(1) secret; h > 0: exactly h coefficients in {-1, +1}
SecretKey *keygen_sk(Ctx *c, u64 seed, int h = 0);
// relin_level < 0: the relinearisation key at the top level
EvalKey *keygen_evk(Ctx *c, const SecretKey *sk, u64 seed, int relin_level = -1);
// one key per step, generated up to levels[i] (empty: the top level); a key
// already present at a level >= the requested one is kept
void keygen_rot(Ctx *c, const SecretKey *sk, EvalKey *evk, const std::vector<int> &steps,
                const std::vector<int> &levels = {});
// the same for Galois elements (X -> X^g, g odd, < 2N; the key id is g)
void keygen_galois(Ctx *c, const SecretKey *sk, EvalKey *evk, const std::vector<u64> &gals,
                   const std::vector<int> &levels = {});
Ciphertext *encrypt_pt(Ctx *c, const EvalKey *evk, const Plaintext *pt, u64 seed);
void decrypt_slots(Ctx *c, const SecretKey *sk, const Ciphertext *ct, double *h_out, int n_slots);
// decrypt into a device buffer, stream-ordered, no synchronisation
void decrypt_slots_device(Ctx *c, const SecretKey *sk, const Ciphertext *ct, double *d_out, int n_slots);
// the rotation key of a Galois element, for a key switch at `level` (HELRM_E_NOKEY if
// missing or generated below that level)
const SwitchKey *rot_key(const EvalKey *evk, u64 galois, int level);
const SwitchKey *relin_key(const EvalKey *evk, int level);

// ------------------------------------------------------ matvec (linear.cu)
struct PtMatrix : Handle {
    Ctx *ctx;
    int in_pad = 0, out_pad = 0, D = 0, n1 = 0, n2 = 0, level = 0;
    double pt_scale = 0, out_scale = 0;
    std::vector<std::pair<int, int>> folds;   // fold levels (stride, radix), smallest stride first
    std::vector<std::pair<int, int>> gb;      // non-zero diagonals, (g, b) order
    std::vector<std::unique_ptr<Plaintext>> pts;
    DevMem d_ptrs;                             // device array of diagonal pointers
    DevMem d_gb_index;                         // int [n2][n1] -> index in pts or -1
    PtMatrix(Ctx *c) : Handle(KIND_PTMAT), ctx(c) {}
    std::vector<int> rotations() const;
    void upload_index();
};
PtMatrix *ptmat_prepare(Ctx *c, const double *W, int rows, int cols, int in_pad, int out_pad,
                        int level, double ct_scale, double target_scale);
// the diagonals of W (+ i W_im when W_im != null) encoded at pt_scale; the
// product declares out_scale after its rescale
PtMatrix *ptmat_prepare_scaled(Ctx *c, const double *W, const double *W_im, int rows, int cols, int in_pad,
                               int out_pad, int level, double pt_scale, double out_scale);
Ciphertext *matvec(Ctx *c, const EvalKey *evk, const PtMatrix *m, const Ciphertext *in);
// products of matrices of one shape share their giant steps (linear.cu)
bool same_shape(const PtMatrix *a, const PtMatrix *b);
Ciphertext *matvec_sum(Ctx *c, const EvalKey *evk, const std::vector<const PtMatrix *> &ms,
                       const std::vector<const Ciphertext *> &in);
int pow2ceil(int x);

}  // namespace helrm
