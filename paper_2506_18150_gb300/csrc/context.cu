// context.cu -- parameter set, prime chain, device tables and memory.
//
// Primes (a reading; the paper only fixes Q = prod q_i, appendix "CKKS
// operations"): every prime is NTT-friendly, q = 1 mod 2N; for each requested
// bit size the largest unused such prime below 2^bits is taken, q_0..q_L in
// order, then the K special primes.  Primality: deterministic Miller-Rabin
// with bases 2..37 (exact for 64-bit integers).  The NTT root of each prime is
// psi = g^((q-1)/2N) for the smallest quadratic non-residue g.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "core.cuh"

namespace helrm {

[[noreturn]] void fail(helrm_status code, const std::string &msg) { throw Error{code, msg}; }

// ------------------------------------------------------------ host number theory
static u64 h_mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }
static u64 h_powmod(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = h_mulmod(r, b, m);
        b = h_mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}
static bool h_is_prime(u64 n)
{
    static const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : bases)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        s++;
    }
    for (u64 a : bases) {
        u64 x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = h_mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}
static u64 h_next_prime_below(int bits, u64 two_n, const std::vector<u64> &used)
{
    u64 top = (bits == 64) ? ~0ull : ((1ull << bits) - 1);
    u64 c = (top / two_n) * two_n + 1;
    if (c > top) c -= two_n;
    for (; c > (1ull << (bits - 1)); c -= two_n) {
        if (std::find(used.begin(), used.end(), c) != used.end()) continue;
        if (h_is_prime(c)) return c;
    }
    fail(HELRM_E_PARAM, "not enough NTT-friendly primes of " + std::to_string(bits) + " bits");
}
static u64 h_inv_mod(u64 a, u64 q) { return h_powmod(a, q - 2, q); }
static u64 h_inv64(u64 q)  // q^-1 mod 2^64 (Newton: each step doubles the correct bits)
{
    u64 x = q;  // correct to 3 bits for odd q
    for (int i = 0; i < 6; i++) x *= 2 - q * x;
    return x;
}
static u32 bitrev(u32 x, int bits)
{
    u32 r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

// ------------------------------------------------------------------- memory
void *Ctx::alloc(size_t bytes)
{
    if (bytes == 0) bytes = 8;
    if (mem_cap && mem_in_use + bytes > mem_cap)
        fail(HELRM_E_NOMEM, "memory cap reached (" + std::to_string(mem_in_use + bytes) + " > " +
                                std::to_string(mem_cap) + " bytes)");
    void *p = nullptr;
    cudaError_t e = (alloc_pool && !capturing) ? cudaMallocFromPoolAsync(&p, bytes, alloc_pool, stream)
                                               : cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(HELRM_E_NOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    mem_in_use += bytes;
    mem_peak = std::max(mem_peak, mem_in_use);
    return p;
}
void Ctx::release(void *p, size_t bytes)
{
    if (!p) return;
    cudaFreeAsync(p, stream);
    mem_in_use -= std::min<u64>(mem_in_use, bytes);
}
DevMem::DevMem(Ctx *c, size_t b) : ctx(c), ptr(c->alloc(b)), bytes(b) {}
DevMem::~DevMem()
{
    if (ptr && ctx) ctx->release(ptr, bytes);
}
DevMem &DevMem::operator=(DevMem &&o) noexcept
{
    if (this != &o) {
        if (ptr && ctx) ctx->release(ptr, bytes);
        ctx = o.ctx;
        ptr = o.ptr;
        bytes = o.bytes;
        o.ptr = nullptr;
        o.bytes = 0;
    }
    return *this;
}

Ctx::Side &Ctx::side_of(cudaStream_t home)
{
    auto it = sides.find(home);
    if (it != sides.end()) return it->second;
    Side s;
    CUDA_CHECK(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    CUDA_CHECK(cudaMemPoolCreate(&s.pool, &props));
    u64 thr = ~0ull;   // keep freed blocks for reuse, like the default pool
    CUDA_CHECK(cudaMemPoolSetAttribute(s.pool, cudaMemPoolAttrReleaseThreshold, &thr));
    CUDA_CHECK(cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming));
    CUDA_CHECK(cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming));
    return sides.emplace(home, s).first->second;
}

// With per-kernel timing on, a branch runs inline on the context's stream,
// so that every kernel's pair of events brackets that kernel alone.
Fork::Fork(Ctx *ctx) : c(ctx), home(ctx->stream), side(ctx->prof_on ? nullptr : &ctx->side_of(ctx->stream))
{
    if (!side) return;
    CUDA_CHECK(cudaEventRecord(side->fork, home));
    CUDA_CHECK(cudaStreamWaitEvent(side->stream, side->fork, 0));
}
void Fork::enter()
{
    if (!side) return;
    c->stream = side->stream;
    c->alloc_pool = side->pool;
}
void Fork::leave()
{
    if (!side) return;
    c->stream = home;
    c->alloc_pool = nullptr;
}
void Fork::join()
{
    if (joined || !side) return;
    joined = true;
    CUDA_CHECK(cudaEventRecord(side->join, side->stream));
    CUDA_CHECK(cudaStreamWaitEvent(home, side->join, 0));
}
Fork::~Fork()
{
    if (joined || !side) return;
    // an error unwinds through here: still order the home stream after the branch
    if (cudaEventRecord(side->join, side->stream) == cudaSuccess) cudaStreamWaitEvent(home, side->join, 0);
    cudaGetLastError();
}

cudaEvent_t Ctx::take_event()
{
    // events are recycled once their pair has been read (prof.clear()).
    cudaEvent_t e;
    if (!event_pool.empty()) {
        e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    CUDA_CHECK(cudaEventCreate(&e));
    return e;
}

Ctx::~Ctx()
{
    cudaStreamSynchronize(stream);
    for (auto &r : prof) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (auto e : event_pool) cudaEventDestroy(e);
    modup_tab.clear();
    moddown_tab.clear();
    rescale_tab.clear();
    mdrs_tab.clear();
    d_pinfo = DevMem();
    d_tw_fwd = DevMem();
    d_tw_inv = DevMem();
    d_ninv = DevMem();
    d_fft_tw = DevMem();
    d_slot_of = DevMem();
    d_u_of_slot = DevMem();
    d_pmod_mont = DevMem();
    d_pinv_mont = DevMem();
    d_one_mont = DevMem();
    d_err = DevMem();
    cudaStreamSynchronize(stream);
    for (auto &kv : sides) {
        cudaStreamSynchronize(kv.second.stream);
        cudaStreamDestroy(kv.second.stream);
        cudaEventDestroy(kv.second.fork);
        cudaEventDestroy(kv.second.join);
        cudaMemPoolDestroy(kv.second.pool);   // released once its last block is freed
    }
}

void Ctx::check_device_errors()
{
    int h = 0;
    CUDA_CHECK(cudaMemcpyAsync(&h, d_err.ptr, 4, cudaMemcpyDeviceToHost, stream));
    CUDA_CHECK(cudaStreamSynchronize(stream));
    if (h) {
        CUDA_CHECK(cudaMemsetAsync(d_err.ptr, 0, 8, stream));
        if (h == (int)HELRM_E_TIMEOUT)
            fail(HELRM_E_TIMEOUT, "a bounded device-side wait ran out (the kernel returned early)");
        fail(HELRM_E_INVAL, "an encoded coefficient exceeded 2^62 (scale or slot values too large)");
    }
}

u64 Ctx::galois(int step) const
{
    long long s = ((long long)step % n_slots + n_slots) % n_slots;
    return h_powmod(5, (u64)s, 2ull * N);
}

static void upload(Ctx *c, DevMem &m, const void *h, size_t bytes)
{
    m = DevMem(c, bytes);
    CUDA_CHECK(cudaMemcpyAsync(m.ptr, h, bytes, cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
}

// ----------------------------------------------------- base conversion tables
// Layout (u64): [0] n_src, [1] n_dst, then per src s: q, qinv, hinv_mont, limb;
// per dst k: p, pinv, limb; then hmod[s][k] = (Qs/q_s mod p_k) R mod p_k (the
// conversion constants the fused forward NTT reads, BConvTable::hcol).  The
// factors [(Qs/q_s)^-1]_{q_s} reach the inverse NTT's final scale through
// iscale.
static BConvTable make_bconv(Ctx *c, const std::vector<int> &src_pid, const std::vector<int> &src_limb,
                             const std::vector<int> &dst_pid, const std::vector<int> &dst_limb)
{
    int ns = (int)src_pid.size(), nd = (int)dst_pid.size();
    std::vector<u64> t;
    std::vector<ulonglong2> isc(ns);
    t.push_back(ns);
    t.push_back(nd);
    for (int s = 0; s < ns; s++) {
        u64 q = c->primes[src_pid[s]];
        // Qhat_s = prod_{r != s} q_r, reduced mod q_s
        u64 qh = 1;
        for (int r = 0; r < ns; r++)
            if (r != s) qh = h_mulmod(qh, c->primes[src_pid[r]] % q, q);
        u64 hinv = h_inv_mod(qh, q);
        // the same factor folded into an inverse NTT's final scale
        const u64 w = h_mulmod(h_inv_mod((u64)c->N % q, q), hinv, q);
        isc[s] = make_ulonglong2(w, (u64)(((u128)w << 64) / q));
        t.push_back(q);
        t.push_back(c->pinfo[src_pid[s]].qinv);
        t.push_back(h_mulmod(hinv, c->pinfo[src_pid[s]].rmod, q));   // Montgomery form
        t.push_back((u64)src_limb[s]);
    }
    for (int k2 = 0; k2 < nd; k2++) {
        t.push_back(c->primes[dst_pid[k2]]);
        t.push_back(c->pinfo[dst_pid[k2]].qinv);
        t.push_back((u64)dst_limb[k2]);
    }
    for (int s = 0; s < ns; s++)
        for (int k2 = 0; k2 < nd; k2++) {
            u64 p = c->primes[dst_pid[k2]];
            u64 qh = 1;
            for (int r = 0; r < ns; r++)
                if (r != s) qh = h_mulmod(qh, c->primes[src_pid[r]] % p, p);
            t.push_back(h_mulmod(qh, c->pinfo[dst_pid[k2]].rmod, p));
        }
    BConvTable bt;
    bt.n_src = ns;
    bt.n_dst = nd;
    upload(c, bt.tab, t.data(), t.size() * 8);
    upload(c, bt.iscale, isc.data(), isc.size() * sizeof(ulonglong2));
    return bt;
}

const BConvTable &Ctx::modup_table(int level, int digit)
{
    auto key = std::make_pair(level, digit);
    auto it = modup_tab.find(key);
    if (it != modup_tab.end()) return it->second;
    std::vector<int> sp, sl, dp, dl;
    int lo = digit_lo(digit), hi = digit_hi(digit, level);
    LimbMap m = qmap(level);
    for (int l = 0; l < level + 1 + K; l++) {
        if (l >= lo && l < hi) {
            sp.push_back(m.pid(l));
            sl.push_back(l);
        } else {
            dp.push_back(m.pid(l));
            dl.push_back(l);
        }
    }
    return modup_tab[key] = make_bconv(this, sp, sl, dp, dl);
}

const BConvTable &Ctx::moddown_table(int level)
{
    auto it = moddown_tab.find(level);
    if (it != moddown_tab.end()) return it->second;
    std::vector<int> sp, sl, dp, dl;
    for (int k2 = 0; k2 < K; k2++) {
        sp.push_back(L + 1 + k2);
        sl.push_back(k2);
    }
    for (int l = 0; l <= level; l++) {
        dp.push_back(l);
        dl.push_back(l);
    }
    return moddown_tab[level] = make_bconv(this, sp, sl, dp, dl);
}

// rescale at `level`: per prime i < level: [q_level^-1 mod q_i] in Montgomery form
// (indexed by prime id), then [q_level mod q_i] (plain), then q_level.
const u64 *Ctx::rescale_table(int level)
{
    auto it = rescale_tab.find(level);
    if (it != rescale_tab.end()) return it->second.u();
    std::vector<u64> t(2 * nP() + 1, 0);
    u64 ql = primes[level];
    for (int i = 0; i < level; i++) {
        u64 q = primes[i];
        t[i] = h_mulmod(h_inv_mod(ql % q, q), pinfo[i].rmod, q);
        t[nP() + i] = ql % q;
    }
    t[2 * nP()] = ql;
    DevMem m;
    upload(this, m, t.data(), t.size() * 8);
    return (rescale_tab[level] = std::move(m)).u();
}

// ModDown merged with the rescale at `level` (NttRescale::ep_scal): per prime
// i < level, (P q_level)^-1 R mod q_i, then at nP + i, q_level^-1 R mod q_i.
const u64 *Ctx::moddown_rescale_table(int level)
{
    auto it = mdrs_tab.find(level);
    if (it != mdrs_tab.end()) return it->second.u();
    std::vector<u64> t(2 * nP(), 0);
    const u64 ql = primes[level];
    for (int i = 0; i < level; i++) {
        const u64 q = primes[i];
        u64 P = 1;
        for (int k2 = 0; k2 < K; k2++) P = h_mulmod(P, primes[L + 1 + k2] % q, q);
        const u64 qlinv = h_inv_mod(ql % q, q);
        t[i] = h_mulmod(h_mulmod(h_inv_mod(P, q), qlinv, q), pinfo[i].rmod, q);
        t[nP() + i] = h_mulmod(qlinv, pinfo[i].rmod, q);
    }
    DevMem m;
    upload(this, m, t.data(), t.size() * 8);
    return (mdrs_tab[level] = std::move(m)).u();
}

// -------------------------------------------------------------- creation
Ctx *ctx_create(const helrm_params *p, int device, void *stream)
{
    HCHECK(p, HELRM_E_INVAL, "params is NULL");
    HCHECK(p->log_n >= 10 && p->log_n <= 16, HELRM_E_PARAM, "log_n must be in [10, 16]");
    HCHECK(p->n_q >= 1 && p->n_q <= 32 && p->q_bits, HELRM_E_PARAM, "n_q must be in [1, 32]");
    HCHECK(p->n_p >= 1 && p->n_p <= 8, HELRM_E_PARAM, "n_p must be in [1, 8]");
    HCHECK(p->alpha >= 1 && p->alpha <= 8, HELRM_E_PARAM, "alpha must be in [1, 8]");
    HCHECK(p->p_bits >= 30 && p->p_bits <= 60, HELRM_E_PARAM, "p_bits must be in [30, 60]");
    for (u32 i = 0; i < p->n_q; i++)
        HCHECK(p->q_bits[i] >= 30 && p->q_bits[i] <= 60, HELRM_E_PARAM, "q_bits must be in [30, 60]");
    HCHECK(p->alpha * 61 < 64 + 61 * 8, HELRM_E_PARAM, "alpha too large");

    std::unique_ptr<Ctx> c(new Ctx());
    c->device = device;
    CUDA_CHECK(cudaSetDevice(device));
    CUDA_CHECK(cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device));
    c->stream = (cudaStream_t)stream;
    c->logN = (int)p->log_n;
    c->N = 1 << c->logN;
    c->n_slots = c->N / 2;
    c->L = (int)p->n_q - 1;
    c->K = (int)p->n_p;
    c->alpha = (int)p->alpha;
    c->delta = std::pow(2.0, p->log2_scale);
    u64 two_n = 2ull * c->N;
    for (u32 i = 0; i < p->n_q; i++) c->primes.push_back(h_next_prime_below(p->q_bits[i], two_n, c->primes));
    for (u32 i = 0; i < p->n_p; i++) c->primes.push_back(h_next_prime_below(p->p_bits, two_n, c->primes));
    // alpha * max(q) < 2^64 keeps the base-conversion accumulator's high word below the target prime
    u64 qmax = *std::max_element(c->primes.begin(), c->primes.end());
    HCHECK((u128)qmax * (u128)std::max(c->alpha, c->K) < ((u128)1 << 64), HELRM_E_PARAM,
           "alpha (or K) times the largest prime must stay below 2^64");

    CUDA_CHECK(cudaDeviceGetDefaultMemPool(&c->pool, device));
    u64 thr = ~0ull;
    CUDA_CHECK(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr));

    int nP = c->nP(), N = c->N;
    std::vector<ulonglong2> fwd((size_t)nP * N), inv((size_t)nP * N), ninv(nP);
    std::vector<u64> pw(N);
    for (int i = 0; i < nP; i++) {
        u64 q = c->primes[i];
        PrimeInfo pi;
        pi.q = q;
        pi.qinv = h_inv64(q);
        pi.rmod = (u64)(((u128)1 << 64) % q);
        pi.r2 = h_mulmod(pi.rmod, pi.rmod, q);
        c->pinfo.push_back(pi);
        u64 g = 2;
        while (h_powmod(g, (q - 1) / 2, q) != q - 1) g++;
        u64 psi = h_powmod(g, (q - 1) / two_n, q);
        c->psi.push_back(psi);
        u64 psi_inv = h_inv_mod(psi, q);
        for (int pass = 0; pass < 2; pass++) {
            u64 base = pass == 0 ? psi : psi_inv;
            u64 x = 1;
            for (int e = 0; e < N; e++) {
                pw[e] = x;
                x = h_mulmod(x, base, q);
            }
            auto &tab = pass == 0 ? fwd : inv;
            for (int kk = 0; kk < N; kk++) {
                u64 w = pw[bitrev((u32)kk, c->logN)];
                tab[(size_t)i * N + kk] = make_ulonglong2(w, (u64)(((u128)w << 64) / q));
            }
        }
        u64 ni = h_inv_mod((u64)N % q, q);
        ninv[i] = make_ulonglong2(ni, (u64)(((u128)ni << 64) / q));
    }
    upload(c.get(), c->d_pinfo, c->pinfo.data(), sizeof(PrimeInfo) * nP);
    upload(c.get(), c->d_tw_fwd, fwd.data(), sizeof(ulonglong2) * fwd.size());
    upload(c.get(), c->d_tw_inv, inv.data(), sizeof(ulonglong2) * inv.size());
    upload(c.get(), c->d_ninv, ninv.data(), sizeof(ulonglong2) * nP);

    // FFT tables for encode/decode (FP64)
    std::vector<double2> tw(N / 2);
    const long double PI = 3.14159265358979323846264338327950288L;
    for (int t = 0; t < N / 2; t++) {
        long double ang = -2.0L * PI * (long double)t / (long double)N;
        tw[t] = make_double2((double)std::cos(ang), (double)std::sin(ang));
    }
    upload(c.get(), c->d_fft_tw, tw.data(), sizeof(double2) * tw.size());
    std::vector<int> slot_of(N, -1), u_of_slot(c->n_slots);
    u64 t = 1;
    for (int j = 0; j < c->n_slots; j++) {
        int u = (int)((t - 1) / 2);
        int u2 = (int)((two_n - t - 1) / 2);
        slot_of[u] = j;
        slot_of[u2] = j;
        u_of_slot[j] = u;
        t = t * 5 % two_n;
    }
    upload(c.get(), c->d_slot_of, slot_of.data(), sizeof(int) * N);
    upload(c.get(), c->d_u_of_slot, u_of_slot.data(), sizeof(int) * c->n_slots);

    std::vector<u64> pmod(nP, 0), pinv(nP, 0), one(nP, 0);
    for (int i = 0; i < nP; i++) {
        u64 q = c->primes[i];
        one[i] = c->pinfo[i].rmod;
        if (i > c->L) continue;
        u64 P = 1;
        for (int k2 = 0; k2 < c->K; k2++) P = h_mulmod(P, c->primes[c->L + 1 + k2] % q, q);
        pmod[i] = h_mulmod(P, c->pinfo[i].rmod, q);
        pinv[i] = h_mulmod(h_inv_mod(P, q), c->pinfo[i].rmod, q);
    }
    upload(c.get(), c->d_pmod_mont, pmod.data(), 8 * nP);
    upload(c.get(), c->d_pinv_mont, pinv.data(), 8 * nP);
    upload(c.get(), c->d_one_mont, one.data(), 8 * nP);
    u64 zero = 0;
    upload(c.get(), c->d_err, &zero, 8);
    k::ntt_autotune(c.get());   // launch shapes for this ring degree and GPU
    noalloc_setup(c.get());
    return c.release();
}

}  // namespace helrm
