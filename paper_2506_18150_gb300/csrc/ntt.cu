// ntt.cu -- 64-bit negacyclic NTT / inverse NTT, batched over limbs.
//
// Forward: merged Cooley-Tukey (twiddle psi^brv(m+i) at stage m, block i),
// standard order in, bit-reversed evaluation order out:
// ahat[i] = a(psi^(2 brv(i) + 1)).  Inverse: merged Gentleman-Sande with
// psi^-brv(m+i), then 1/N.  Twiddles carry Shoup quotients; butterflies are
// Harvey's lazy ones (values in [0, 4q) forward, [0, 2q) inverse, q < 2^62),
// corrected once at the end.
//
// N = N1 * N2 runs as two passes, each reading and writing every limb once.
// The first log2(N1) stages pair elements N/2..N2 apart, so each of the N2
// columns (stride N2) is an independent N1-point problem.  The remaining
// log2(N2) stages stay inside contiguous rows of N2.  Within a pass every
// thread keeps 8 elements in registers and applies up to three stages per
// round (a radix-8 step); shared memory is used only to regroup elements
// between rounds, so a 256-point sub-transform costs two barriers.  Loads and
// stores are coalesced: consecutive threads take consecutive columns (column
// pass) or consecutive elements of a row (row pass).
//
// A launch takes a list of limbs, each with its own source, destination and
// prime: the first pass reads the source and writes the destination (so no
// copy is needed before a transform), the second works in place.  A forward
// transform may end with a fused epilogue out = (a - NTT(y)) * c[prime] (+ b)
// (c a Montgomery constant), which is how ModDown and rescale finish.
#include <cstdlib>

#include "butterfly.cuh"

namespace helrm {
namespace {

constexpr int MAX_LIMBS = 128;
inline int tune_bucket(int n_limbs) { return n_limbs <= 4 ? 0 : n_limbs <= 16 ? 1 : n_limbs <= 64 ? 2 : 3; }

struct LimbList {
    int n;
    const u64 *src[MAX_LIMBS];
    u64 *dst[MAX_LIMBS];
    const u64 *ea[MAX_LIMBS];   // epilogue a operand (nullptr: no epilogue)
    const u64 *eb[MAX_LIMBS];   // epilogue addend (nullptr: none)
    u64 *eo[MAX_LIMBS];         // epilogue output
    unsigned short pid[MAX_LIMBS];
};

// Per-limb extras of a column pass (NttLimb::scal / fbc_*), passed only to
// the instances that use them so that plain launches keep a smaller argument
// block.  A conversion has at most FBC_MAX source limbs (alpha and K are 3).
constexpr int FBC_MAX = 4;
struct XList {
    const ulonglong2 *scal[MAX_LIMBS];   // inverse: final scale (null: N^-1)
    const u64 *fh[MAX_LIMBS];            // forward: conversion constants, stride fhs
    const u64 *rs_u[MAX_LIMBS];          // forward, merged rescale: top limb of the half (coefficients)
    const u64 *rs_add[MAX_LIMBS];        //   and of its addend (null: none)
    unsigned short fhs[MAX_LIMBS];
    unsigned char fn[MAX_LIMBS];         // forward: source limbs (0: plain input)
    // merged rescale, uniform over the launch: the conversion constants of the
    // dropped prime q_l (stride hls), its prime id, and per prime id P R mod q
    // and q_l mod q
    const u64 *hl;
    int hls, lp;
    const u64 *pmod, *qlmod, *pinv;
};
// Epilogue constants of a forward transform's last pass: eo = (ea - NTT(y)) *
// scal[pid] + eb, the addend scaled by scal[add_off + pid] when add_off > 0.
struct Ep {
    const u64 *scal = nullptr;
    int add_off = 0;
};
template <bool XL>
struct XArg {
    XList x;
};
template <>
struct XArg<false> {
};

enum Mode { M_LAZY = 0, M_SCALE = 1, M_REDUCE = 2 };

// One pass over sub-transforms of P = 2^LOGP points.
// COLS: sub-transform g is column g of the limb, elements r*N2 + g.
// ROWS: sub-transform g is row g, elements g*N2 + x.
// Twiddle of local stage s, local block lb: tw[((bm + seg) << s) + lb], with
// bm = 1, seg = 0 for the column pass and bm = N1, seg = row for the row pass.
// mode: M_LAZY leaves the lazy range (first pass), M_SCALE multiplies by 1/N
// (last inverse pass), M_REDUCE reduces to [0, q) (last forward pass) and
// applies the epilogue where the limb has one.
// FIXN > 0: the ring degree is 2^FIXN and the tile holds 2^FIXG sub-transforms,
// both compile-time constants (the production sizes), so every shared- and
// global-memory address is a per-thread base plus an immediate offset; 0: the
// arguments logN / logG are used (every other size).
// Register budget of the fixed-size instances with tiles of 4 or 8
// sub-transforms (128, 256 threads): 48 registers, i.e. 40 resident warps per
// SM instead of 32, without spills; every other instance is left to the
// compiler under the 512-thread bound (it settles at 56-64 registers).
// EPT = 4 elements per thread (fixed-size instances only): radix-4 rounds,
// twice the threads per sub-transform and half the serial work per thread,
// which shortens launches that carry few limbs; up to 64 registers.
#define NTT_MAX_THREADS(FIXN, FIXG, EPT) ((FIXN) && (FIXG) >= 2 ? ((256 / (EPT)) << (FIXG)) : 512)
#define NTT_MIN_BLOCKS(FIXN, FIXG, EPT) \
    ((FIXN) && (FIXG) >= 2 ? 65536 / (((256 / (EPT)) << (FIXG)) * ((EPT) == 8 ? 48 : 64)) : 0)

// XL (column passes only): the per-limb extras of XList apply -- a forward
// first pass computes its input as a fast base conversion of fn source limbs
// on load (the 128-bit multiply-accumulate and the one reduction of the
// stand-alone conversion kernel, so the values are identical); an inverse
// last pass scales by its own constant.
template <int LOGP, bool COLS, bool INV, int FIXN = 0, int FIXG = 0, bool XL = false, int EPT = 8>
__global__ void __launch_bounds__(NTT_MAX_THREADS(FIXN, FIXG, EPT), NTT_MIN_BLOCKS(FIXN, FIXG, EPT)) k_ntt_pass(int first, int logN_arg, int logG_arg, LimbList list,
                                                   const ulonglong2 *__restrict__ tw_all,
                                                   const ulonglong2 *__restrict__ ninv,
                                                   const PrimeInfo *__restrict__ pinfo, int mode, const Ep ep,
                                                   const XArg<XL> xa)
{
    constexpr int P = 1 << LOGP;
    constexpr int TPS = P / EPT;            // threads per sub-transform (EPT elements each)
    constexpr int RB = EPT >= 8 ? 3 : 2;    // stages per round
    extern __shared__ u64 sm[];
    const int logN = FIXN ? FIXN : logN_arg;
    const int logG = FIXN ? FIXG : logG_arg;
    const int N = 1 << logN;
    const int logN1 = logN / 2;
    const int N2 = N >> logN1;
    const int G = 1 << logG;                // sub-transforms per CTA
    const int y = blockIdx.y;
    const int pid = list.pid[y];
    const ulonglong2 *tw = tw_all + (size_t)pid * N;
    const u64 *in = first ? list.src[y] : list.dst[y];
    u64 *out = list.dst[y];
    const u64 *ea = list.ea[y];
    const u64 *eb = list.eb[y];
    u64 *eo = list.eo[y];
    const int tid = threadIdx.x;
    // thread -> (sub-transform g, lane tt); for COLS, g varies fastest so a
    // warp reads consecutive columns of one row.
    int g, tt;
    if (COLS) {
        g = tid & (G - 1);
        tt = tid >> logG;
    } else {
        tt = tid & (TPS - 1);
        g = tid / TPS;
    }
    const int gglob = blockIdx.x * G + g;   // column index (COLS) or row index (ROWS)
    const int bm = COLS ? 1 : (1 << logN1);
    const int seg = COLS ? 0 : gglob;

    // The prime and the twiddles do not depend on earlier kernels, so they are
    // fetched before the grid-dependency wait, overlapping the previous
    // kernel: the prime constants into registers, and the 128-byte lines of
    // this sub-transform's twiddles (the run of 2^s entries at (bm + seg) << s
    // for each local stage s; lane tt takes entries [8 tt, 8 tt + 8) of each
    // run) into L2.  The column pass's set is shared, so only its g = 0 lanes
    // fetch it.
    const PrimeInfo pi = pinfo[pid];
    int fn = 0;                 // fused conversion: source limbs and their constants
    u64 hk[FBC_MAX], hl[FBC_MAX];
    const u64 *rs_u = nullptr, *rs_add = nullptr;
    PrimeInfo pl;
    u64 pl_pinv = 0, pmod_q = 0, qlmod_q = 0;
    ulonglong2 xs = make_ulonglong2(0, 0);
    if constexpr (XL) {
        if (!INV) {
            fn = xa.x.fn[y];
            const u64 *fh = xa.x.fh[y];
            const int hs = xa.x.fhs[y];
#pragma unroll
            for (int s = 0; s < FBC_MAX; s++) hk[s] = s < fn ? fh[s * hs] : 0;
            rs_u = xa.x.rs_u[y];
            if (rs_u) {   // merged rescale: the dropped prime's constants
                rs_add = xa.x.rs_add[y];
#pragma unroll
                for (int s = 0; s < FBC_MAX; s++) hl[s] = s < fn ? xa.x.hl[s * xa.x.hls] : 0;
                pl = pinfo[xa.x.lp];
                pl_pinv = xa.x.pinv[xa.x.lp];
                pmod_q = xa.x.pmod[pid];
                qlmod_q = xa.x.qlmod[pid];
            }
        } else if (xa.x.scal[y]) {
            xs = *xa.x.scal[y];
        }
    }
    if (!COLS || g == 0) {
#pragma unroll
        for (int s = 0; s < LOGP; s++)
            for (int e = tt * 8; e < (1 << s); e += TPS * 8) {
                const ulonglong2 *line = tw + ((size_t)(bm + seg) << s) + e;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
            }
    }
    pdl_begin();
    const u64 q = pi.q;
    const u64 q2 = 2 * q;
    auto gaddr = [&](int e) -> size_t {
        return COLS ? (size_t)e * N2 + gglob : (size_t)gglob * N2 + e;
    };
    // padded shared-memory index pad(x) = x + x/16 of element e, split into a
    // per-thread part and a part that depends on e only (a constant once the
    // rounds are unrolled and G is fixed): for COLS, x = e G + g with g < G, so
    // x/16 = (e G)/16 + (G > 16 ? g/16 : 0); for ROWS, x = g P + e with P a
    // multiple of 16, so x/16 = (g P)/16 + e/16
    const int sbase = COLS ? (G <= 16 ? g : g + (g >> 4)) : (g * P + ((g * P) >> 4));
    auto saddr = [&](int e) -> int { return COLS ? e * G + ((e * G) >> 4) + sbase : e + (e >> 4) + sbase; };

    u64 v[EPT];
    // rounds of up to RB stages; forward goes first-to-last, inverse last-to-first
    constexpr int NR = (LOGP + RB - 1) / RB;
#pragma unroll
    for (int rr = 0; rr < NR; rr++) {
        const int rho = INV ? NR - 1 - rr : rr;
        const int s0 = RB * rho;
        const int r = (s0 + RB <= LOGP) ? RB : LOGP - s0;
        const int T = P >> (s0 + r);        // spacing of a group's members
        const int gs = 1 << r;              // group size
        const int ng = EPT / gs;            // groups per thread
        // element index of member k of this thread's group qg
        auto elem = [&](int qg, int k) {
            const int gam = tt + qg * TPS;  // group index
            const int blk = gam / T, boff = gam % T;
            return blk * (T * gs) + boff + k * T;
        };
        if (rr == 0) {
            if (XL && !INV && fn) {
#pragma unroll
                for (int qg = 0; qg < ng; qg++)
#pragma unroll
                    for (int k = 0; k < gs; k++) {
                        const size_t a = gaddr(elem(qg, k));
                        Acc128 acc;
                        u64 ts[FBC_MAX];
#pragma unroll
                        for (int s = 0; s < FBC_MAX; s++)
                            if (s < fn) {
                                ts[s] = in[(size_t)s * N + a];
                                acc.mac(ts[s], hk[s], q);
                            }
                        if (rs_u) {
                            // the ModDown result's top limb in coefficient form,
                            // x = (u_l - FBC_l) P^-1 (+ add_l) mod q_l, centred and
                            // taken mod q: P r joins the conversion before the REDC
                            Acc128 al;
#pragma unroll
                            for (int s = 0; s < FBC_MAX; s++)
                                if (s < fn) al.mac(ts[s], hl[s], pl.q);
                            u64 x = mont_mul(sub_mod(rs_u[a], al.reduce(pl.q, pl.qinv), pl.q), pl_pinv, pl.q, pl.qinv);
                            if (rs_add) x = add_mod(x, rs_add[a], pl.q);
                            const u64 xm = x < q ? x : x % q;
                            acc.mac(x <= ((pl.q - 1) >> 1) ? xm : sub_mod(xm, qlmod_q, q), pmod_q, q);
                        }
                        v[qg * gs + k] = acc.reduce(q, pi.qinv);
                    }
            } else {
#pragma unroll
                for (int qg = 0; qg < ng; qg++)
#pragma unroll
                    for (int k = 0; k < gs; k++) v[qg * gs + k] = in[gaddr(elem(qg, k))];
            }
        } else {
            __syncthreads();
#pragma unroll
            for (int qg = 0; qg < ng; qg++)
#pragma unroll
                for (int k = 0; k < gs; k++) v[qg * gs + k] = sm[saddr(elem(qg, k))];
        }
        // The group's members all lie in block blk of stage s0, so at stage
        // s0 + u the butterfly of member k1 uses local block
        // (blk << u) + (k1 >> (r - u)): 2^u distinct twiddles, loaded once.
#pragma unroll
        for (int qg = 0; qg < ng; qg++) {
            u64 *x = v + qg * gs;
            const int blk = (tt + qg * TPS) / T;
#pragma unroll
            for (int uu = 0; uu < r; uu++) {
                const int u = INV ? r - 1 - uu : uu;
                const int s = s0 + u;
                const int half = gs >> (u + 1);
                const ulonglong2 *twb = tw + (((bm + seg) << s) + (blk << u));
                ulonglong2 wv[4];
#pragma unroll
                for (int j = 0; j < (1 << u); j++) wv[j] = twb[j];
#pragma unroll
                for (int k1 = 0; k1 < gs; k1++) {
                    if (k1 & half) continue;
                    const ulonglong2 w = wv[k1 >> (r - u)];
                    if (!INV)
                        bfly_ct(x[k1], x[k1 + half], w.x, w.y, q, q2);
                    else
                        bfly_gs(x[k1], x[k1 + half], w.x, w.y, q, q2);
                }
            }
        }
        if (rr + 1 < NR) {
            if (rr > 0) __syncthreads();    // everyone has read the previous round's layout
#pragma unroll
            for (int qg = 0; qg < ng; qg++)
#pragma unroll
                for (int k = 0; k < gs; k++) sm[saddr(elem(qg, k))] = v[qg * gs + k];
        } else {
            ulonglong2 ni = make_ulonglong2(0, 0);
            u64 ec = 0, ec2 = 0;
            if (mode == M_SCALE) ni = (XL && INV && xs.x) ? xs : ninv[pid];
            if (mode == M_REDUCE && ea) {
                ec = ep.scal[pid];
                if (ep.add_off) ec2 = ep.scal[ep.add_off + pid];
            }
#pragma unroll
            for (int qg = 0; qg < ng; qg++)
#pragma unroll
                for (int k = 0; k < gs; k++) {
                    u64 z = v[qg * gs + k];
                    const size_t a = gaddr(elem(qg, k));
                    if (mode == M_SCALE) {
                        out[a] = shoup_mul(z, ni.x, ni.y, q);
                    } else if (mode == M_REDUCE) {
                        z = csub(csub(z, q2), q);
                        if (ea) {
                            u64 w = mont_mul(sub_mod(ea[a], z, q), ec, q, pi.qinv);
                            if (eb) w = add_mod(w, ep.add_off ? mont_mul(eb[a], ec2, q, pi.qinv) : eb[a], q);
                            eo[a] = w;
                        } else
                            out[a] = z;
                    } else {
                        out[a] = z;
                    }
                }
        }
    }
}

template <int LOGP, bool COLS, bool INV, int FIXN, int FIXG, bool XL, int EPT = 8>
void launch_kernel(Ctx *c, dim3 grid, int threads, size_t smem, const LimbList &ll, int first, int logG, int mode,
                   const Ep &ep_scal, const XArg<XL> &xa)
{
    const ulonglong2 *tw = INV ? c->d_tw_inv.as<ulonglong2>() : c->d_tw_fwd.as<ulonglong2>();
    launch(c, k_ntt_pass<LOGP, COLS, INV, FIXN, FIXG, XL, EPT>, grid, threads, smem, first, c->logN, logG, ll, tw,
           c->d_ninv.as<ulonglong2>(), c->d_pinfo.as<PrimeInfo>(), mode, ep_scal, xa);
}

template <int LOGP, bool COLS, bool INV, bool XL>
void launch_pass(Ctx *c, const LimbList &ll, int n_sub, int first, int mode, const Ep &ep_scal, const XArg<XL> &xa)
{
    constexpr int P = 1 << LOGP;
    // sub-transforms per CTA: as many as fit the tuned tile, fewer when the
    // batch is small so the grid still covers the SMs (columns keep >= 4
    // consecutive words per row for coalescing)
    const Ctx::NttTune &tu = c->ntt_tune[tune_bucket(ll.n)];
    int G = std::max(1, std::min(tu.tile / P, n_sub));
    const int gmin = COLS ? 4 : 1;
    while (G > gmin && (long)(n_sub / G) * ll.n < (long)tu.mult * c->n_sms) G /= 2;
    int logG = 0;
    while ((1 << logG) < G) logG++;
    const size_t smem = (size_t)(G * P + (G * P >> 4) + 1) * 8;
    dim3 grid(n_sub / G, ll.n);
    // N = 2^16 (both passes 256-point): instances with the tile width fixed,
    // with 8 or 4 elements per thread
    if constexpr (LOGP == 8) {
        if (c->logN == 16 && tu.ept == 4) {
            const int t4 = G * P / 4;
            switch (logG) {
            case 0: launch_kernel<8, COLS, INV, 16, 0, XL, 4>(c, grid, t4, smem, ll, first, logG, mode, ep_scal, xa); return;
            case 1: launch_kernel<8, COLS, INV, 16, 1, XL, 4>(c, grid, t4, smem, ll, first, logG, mode, ep_scal, xa); return;
            case 2: launch_kernel<8, COLS, INV, 16, 2, XL, 4>(c, grid, t4, smem, ll, first, logG, mode, ep_scal, xa); return;
            case 3: launch_kernel<8, COLS, INV, 16, 3, XL, 4>(c, grid, t4, smem, ll, first, logG, mode, ep_scal, xa); return;
            default: break;
            }
        }
    }
    const int threads = G * P / 8;
    if constexpr (LOGP == 8) {
        if (c->logN == 16) {
            switch (logG) {
            case 0: launch_kernel<8, COLS, INV, 16, 0, XL>(c, grid, threads, smem, ll, first, logG, mode, ep_scal, xa); return;
            case 1: launch_kernel<8, COLS, INV, 16, 1, XL>(c, grid, threads, smem, ll, first, logG, mode, ep_scal, xa); return;
            case 2: launch_kernel<8, COLS, INV, 16, 2, XL>(c, grid, threads, smem, ll, first, logG, mode, ep_scal, xa); return;
            case 3: launch_kernel<8, COLS, INV, 16, 3, XL>(c, grid, threads, smem, ll, first, logG, mode, ep_scal, xa); return;
            default: break;
            }
        }
    }
    launch_kernel<LOGP, COLS, INV, 0, 0, XL>(c, grid, threads, smem, ll, first, logG, mode, ep_scal, xa);
}

template <bool COLS, bool INV, bool XL>
void dispatch(Ctx *c, int logp, const LimbList &ll, int n_sub, int first, int mode, const Ep &ep_scal,
              const XArg<XL> &xa)
{
    switch (logp) {
    case 5: launch_pass<5, COLS, INV, XL>(c, ll, n_sub, first, mode, ep_scal, xa); break;
    case 6: launch_pass<6, COLS, INV, XL>(c, ll, n_sub, first, mode, ep_scal, xa); break;
    case 7: launch_pass<7, COLS, INV, XL>(c, ll, n_sub, first, mode, ep_scal, xa); break;
    case 8: launch_pass<8, COLS, INV, XL>(c, ll, n_sub, first, mode, ep_scal, xa); break;
    default: fail(HELRM_E_PARAM, "unsupported NTT size");
    }
}

// both passes of one launch list; xl (may be null) holds the column pass's
// per-limb extras: the forward transform's first pass, the inverse's last
void run_list(Ctx *c, const LimbList &ll, bool inverse, const Ep &ep_scal, const XArg<true> *xl = nullptr)
{
    const int logN = c->logN, logN1 = logN / 2, logN2 = logN - logN1;
    const int N1 = 1 << logN1, N2 = 1 << logN2;
    const XArg<false> none;
    const Ep no_ep;
    if (!inverse) {
        if (xl)
            dispatch<true, false, true>(c, logN1, ll, N2, 1, M_LAZY, no_ep, *xl);
        else
            dispatch<true, false, false>(c, logN1, ll, N2, 1, M_LAZY, no_ep, none);
        dispatch<false, false, false>(c, logN2, ll, N1, 0, M_REDUCE, ep_scal, none);
    } else {
        dispatch<false, true, false>(c, logN2, ll, N1, 1, M_LAZY, no_ep, none);
        if (xl)
            dispatch<true, true, true>(c, logN1, ll, N2, 0, M_SCALE, no_ep, *xl);
        else
            dispatch<true, true, false>(c, logN1, ll, N2, 0, M_SCALE, no_ep, none);
    }
    c->launches += 2;
    CUDA_CHECK(cudaGetLastError());
}

}  // namespace

namespace k {

// rs (forward only, may be null): the launch is a merged ModDown + rescale
static void ntt_run_impl(Ctx *c, const std::vector<NttLimb> &limbs, bool inverse, const Ep &ep,
                         const NttRescale *rs)
{
    if (limbs.empty()) return;
    KTimer kt(c, "ntt", 16.0 * c->N * limbs.size());   // algorithmic: each limb read and written once
    std::unique_ptr<XArg<true>> xl;
    for (size_t b = 0; b < limbs.size(); b += MAX_LIMBS) {
        LimbList ll;
        ll.n = (int)std::min<size_t>(MAX_LIMBS, limbs.size() - b);
        bool extras = rs != nullptr;
        for (int i = 0; i < ll.n; i++) {
            const NttLimb &x = limbs[b + i];
            ll.src[i] = x.src;
            ll.dst[i] = x.dst;
            ll.ea[i] = x.ea;
            ll.eb[i] = x.eb;
            ll.eo[i] = x.eo;
            ll.pid[i] = (unsigned short)x.pid;
            extras |= (inverse ? x.scal != nullptr : x.fbc_n > 0);
        }
        if (extras) {
            if (!xl) xl.reset(new XArg<true>());
            for (int i = 0; i < ll.n; i++) {
                const NttLimb &x = limbs[b + i];
                HCHECK(x.fbc_n >= 0 && x.fbc_n <= FBC_MAX && x.fbc_hs >= 0 && x.fbc_hs < 65536, HELRM_E_PARAM,
                       "fused base conversion: at most 4 source limbs");
                HCHECK(!x.fbc_n || x.src != x.dst, HELRM_E_PARAM, "fused base conversion cannot run in place");
                HCHECK(!x.rs_u || (rs && x.fbc_n), HELRM_E_PARAM, "a merged rescale needs a fused conversion");
                xl->x.scal[i] = inverse ? x.scal : nullptr;
                xl->x.fn[i] = (unsigned char)(inverse ? 0 : x.fbc_n);
                xl->x.fh[i] = x.fbc_h;
                xl->x.fhs[i] = (unsigned short)x.fbc_hs;
                xl->x.rs_u[i] = inverse ? nullptr : x.rs_u;
                xl->x.rs_add[i] = inverse ? nullptr : x.rs_add;
            }
            if (rs) {
                xl->x.hl = rs->hl;
                xl->x.hls = rs->hls;
                xl->x.lp = rs->lp;
                xl->x.pmod = rs->pmod;
                xl->x.qlmod = rs->qlmod;
                xl->x.pinv = rs->pinv;
            }
        }
        run_list(c, ll, inverse, ep, extras ? xl.get() : nullptr);
    }
}

void ntt_run(Ctx *c, const std::vector<NttLimb> &limbs, bool inverse, const u64 *ep_scal)
{
    Ep ep;
    ep.scal = ep_scal;
    ntt_run_impl(c, limbs, inverse, ep, nullptr);
}

void ntt_run_rescale(Ctx *c, const std::vector<NttLimb> &limbs, const NttRescale &rs)
{
    Ep ep;
    ep.scal = rs.ep_scal;
    ep.add_off = rs.add_off;
    ntt_run_impl(c, limbs, false, ep, &rs);
}

// Contiguous limbs described by a LimbMap, in place; the launch list is built
// on the stack (no heap or device allocation on this path).
void ntt_map_noheap(Ctx *c, u64 *data, int n_limbs, LimbMap map, bool inverse)
{
    if (n_limbs <= 0) return;
    KTimer kt(c, "ntt", 16.0 * c->N * n_limbs);
    const size_t N = (size_t)c->N;
    for (int b = 0; b < n_limbs; b += MAX_LIMBS) {
        LimbList ll;
        ll.n = std::min(MAX_LIMBS, n_limbs - b);
        for (int i = 0; i < ll.n; i++) {
            ll.src[i] = ll.dst[i] = data + (size_t)(b + i) * N;
            ll.ea[i] = nullptr;
            ll.eb[i] = nullptr;
            ll.eo[i] = nullptr;
            ll.pid[i] = (unsigned short)map.pid(b + i);
        }
        run_list(c, ll, inverse, Ep());
    }
}

void ntt_autotune(Ctx *c)
{
    const char *env = getenv("HELRM_NTT_AUTOTUNE");
    if (env && env[0] == '0') return;   // keep the default shapes
    const int N = c->N, n_max = 128;
    const int tiles[] = {512, 1024, 2048};
    const int mults[] = {1, 2, 4, 8};
    const char *ept_env = getenv("HELRM_NTT_EPT");   // 4 or 8: tune with that width only
    std::vector<int> epts = {8, 4};
    if (ept_env && (atoi(ept_env) == 8 || atoi(ept_env) == 4)) epts = {atoi(ept_env)};
    const int sizes[4] = {2, 8, 32, 128};   // a representative launch of each bucket
    DevMem buf(c, (size_t)n_max * N * 8);
    CUDA_CHECK(cudaMemsetAsync(buf.ptr, 0, (size_t)n_max * N * 8, c->stream));
    cudaEvent_t e0, e1;
    CUDA_CHECK(cudaEventCreate(&e0));
    CUDA_CHECK(cudaEventCreate(&e1));
    const bool prof = c->prof_on;
    c->prof_on = false;
    for (int bk = 0; bk < 4; bk++) {
        const int n = sizes[bk];
        std::vector<NttLimb> v;
        for (int l = 0; l < n; l++) {
            u64 *p = buf.u() + (size_t)l * N;
            v.push_back({p, p, 1 + l % std::max(c->L, 1), nullptr, nullptr, nullptr});
        }
        float best = 1e30f;
        Ctx::NttTune win = c->ntt_tune[bk];
        for (int e : epts)
        for (int t : tiles)
            for (int m : mults) {
                if (e != 8 && N != 65536) continue;   // 4 per thread: the N = 2^16 instances only
                c->ntt_tune[bk] = {t, m, e};
                ntt_run(c, v, false, nullptr);   // warm-up
                ntt_run(c, v, true, nullptr);
                CUDA_CHECK(cudaEventRecord(e0, c->stream));
                for (int r = 0; r < 3; r++) {
                    ntt_run(c, v, false, nullptr);
                    ntt_run(c, v, true, nullptr);
                }
                CUDA_CHECK(cudaEventRecord(e1, c->stream));
                CUDA_CHECK(cudaEventSynchronize(e1));
                float ms = 0;
                CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best * 0.98f) {   // prefer the earlier (smaller) shape unless clearly faster
                    best = ms;
                    win = {t, m, e};
                }
            }
        c->ntt_tune[bk] = win;
    }
    c->prof_on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
}

void ntt_list(Ctx *c, u64 *base, const std::vector<std::pair<u32, int>> &limbs, bool inverse)
{
    std::vector<NttLimb> v;
    v.reserve(limbs.size());
    for (auto &x : limbs) {
        u64 *p = base + (size_t)x.first * c->N;
        v.push_back({p, p, x.second, nullptr, nullptr, nullptr});
    }
    ntt_run(c, v, inverse, nullptr);
}

void ntt_fwd(Ctx *c, u64 *data, int n_limbs, LimbMap map)
{
    std::vector<NttLimb> v;
    for (int l = 0; l < n_limbs; l++) {
        u64 *p = data + (size_t)l * c->N;
        v.push_back({p, p, map.pid(l), nullptr, nullptr, nullptr});
    }
    ntt_run(c, v, false, nullptr);
}

void ntt_inv(Ctx *c, u64 *data, int n_limbs, LimbMap map)
{
    std::vector<NttLimb> v;
    for (int l = 0; l < n_limbs; l++) {
        u64 *p = data + (size_t)l * c->N;
        v.push_back({p, p, map.pid(l), nullptr, nullptr, nullptr});
    }
    ntt_run(c, v, true, nullptr);
}

}  // namespace k
}  // namespace helrm
