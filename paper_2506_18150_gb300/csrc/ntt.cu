// ntt.cu -- 64-bit negacyclic NTT / inverse NTT, batched over limbs.
//
// Forward: merged Cooley-Tukey (twiddle psi^brv(m+i) at stage m, block i),
// standard order in, bit-reversed evaluation order out:
// ahat[i] = a(psi^(2 brv(i) + 1)).  Inverse: merged Gentleman-Sande with
// psi^-brv(m+i), then 1/N.  Twiddles carry Shoup quotients.
//
// N = N1 * N2 runs as two passes, each reading and writing every limb once.
// The first log2(N1) stages pair elements N/2..N2 apart, so each of the N2
// columns (stride N2) is an independent N1-point problem.  The remaining
// log2(N2) stages stay inside contiguous rows of N2.  Within a pass every
// thread keeps 8 elements in registers and applies up to three stages per
// round (a radix-8 step); shared memory is used only to regroup elements
// between rounds, so a 256-point sub-transform costs two barriers.  Loads and
// stores are coalesced: consecutive threads take consecutive columns (column
// pass) or consecutive elements of a row (row pass).  A launch takes any list
// of limbs (offset, prime), so a whole ModUp or ModDown is one transform.
#include "core.cuh"

namespace helrm {
namespace {

constexpr int MAX_LIMBS = 256;
constexpr int TILE = 4096;   // words per CTA (32 KB of data)

struct LimbList {
    int n;
    u32 off[MAX_LIMBS];   // limb offset from the base pointer, in limbs
    unsigned short pid[MAX_LIMBS];
};

__device__ __forceinline__ int pad(int e) { return e + (e >> 4); }

// Harvey's lazy butterflies (all values < 4q < 2^64 since every q < 2^62).
// Shoup product without its final correction: a * w mod q in [0, 2q).
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q) { return a * w - mulhi64(a, wp) * q; }
// forward (Cooley-Tukey): x0, x1 in [0, 4q) -> [0, 4q)
__device__ __forceinline__ void bfly_ct(u64 &x0, u64 &x1, u64 w, u64 wp, u64 q, u64 q2)
{
    u64 a = x0 >= q2 ? x0 - q2 : x0;
    u64 t = shoup_lazy(x1, w, wp, q);
    x0 = a + t;
    x1 = a - t + q2;
}
// inverse (Gentleman-Sande): x0, x1 in [0, 2q) -> [0, 2q)
__device__ __forceinline__ void bfly_gs(u64 &x0, u64 &x1, u64 w, u64 wp, u64 q, u64 q2)
{
    u64 s = x0 + x1;
    s = s >= q2 ? s - q2 : s;
    u64 t = x0 - x1 + q2;
    x0 = s;
    x1 = shoup_lazy(t, w, wp, q);
}
// [0, 4q) -> [0, q)
__device__ __forceinline__ u64 reduce4(u64 x, u64 q, u64 q2)
{
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

// One pass of the forward transform over sub-transforms of P = 2^LOGP points.
// COLS: sub-transform g is column c0+g of the limb, elements r*N2 + c.
// ROWS: sub-transform g is row r0+g, elements (r0+g)*N2 + x.
// Twiddle of local stage s, local block lb: tw[((bm + seg) << s) + lb], with
// bm = 1, seg = 0 for the column pass and bm = N1, seg = row for the row pass.
template <int LOGP, bool COLS, bool INV>
__global__ void __launch_bounds__(512) k_ntt_pass(u64 *data, int logN, int logG, LimbList list,
                                                   const ulonglong2 *__restrict__ tw_all,
                                                   const ulonglong2 *__restrict__ ninv,
                                                   const PrimeInfo *__restrict__ pinfo, int scale_out)
{
    constexpr int P = 1 << LOGP;
    constexpr int TPS = P / 8;              // threads per sub-transform
    extern __shared__ u64 sm[];
    const int N = 1 << logN;
    const int logN1 = logN / 2;
    const int N2 = N >> logN1;
    const int G = 1 << logG;                // sub-transforms per CTA
    const int pid = list.pid[blockIdx.y];
    const u64 q = pinfo[pid].q;
    const u64 q2 = 2 * q;
    const ulonglong2 *tw = tw_all + (size_t)pid * N;
    u64 *a = data + (size_t)list.off[blockIdx.y] * N;
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
    auto gaddr = [&](int e) -> size_t {
        return COLS ? (size_t)e * N2 + gglob : (size_t)gglob * N2 + e;
    };
    auto saddr = [&](int e) -> int { return COLS ? pad(e * G + g) : pad(g * P + e); };

    u64 v[8];
    // rounds of up to three stages; forward goes first-to-last, inverse last-to-first
    constexpr int NR = (LOGP + 2) / 3;
    _Pragma("unroll") for (int rr = 0; rr < NR; rr++) {
        const int rho = INV ? NR - 1 - rr : rr;
        const int s0 = 3 * rho;
        const int r = (s0 + 3 <= LOGP) ? 3 : LOGP - s0;
        const int T = P >> (s0 + r);        // spacing of a group's members
        const int gs = 1 << r;              // group size
        const int ng = 8 / gs;              // groups per thread
        // element index of member k of this thread's group qg
        auto elem = [&](int qg, int k) {
            const int gam = tt + qg * TPS;  // group index
            const int blk = gam / T, boff = gam % T;
            return blk * (T * gs) + boff + k * T;
        };
        if (rr == 0) {
            _Pragma("unroll") for (int qg = 0; qg < ng; qg++)
                _Pragma("unroll") for (int k = 0; k < gs; k++) v[qg * gs + k] = a[gaddr(elem(qg, k))];
        } else {
            __syncthreads();
            _Pragma("unroll") for (int qg = 0; qg < ng; qg++)
                _Pragma("unroll") for (int k = 0; k < gs; k++) v[qg * gs + k] = sm[saddr(elem(qg, k))];
        }
        _Pragma("unroll") for (int qg = 0; qg < ng; qg++) {
            u64 *x = v + qg * gs;
            const int e0 = elem(qg, 0);
            if (!INV) {
                _Pragma("unroll") for (int u = 0; u < r; u++) {
                    const int s = s0 + u;
                    const int half = gs >> (u + 1);
                    _Pragma("unroll") for (int k1 = 0; k1 < gs; k1++) {
                        if (k1 & half) continue;
                        const int lb = (e0 + k1 * T) >> (LOGP - s);
                        const ulonglong2 w = tw[((bm + seg) << s) + lb];
                        bfly_ct(x[k1], x[k1 + half], w.x, w.y, q, q2);
                    }
                }
            } else {
                _Pragma("unroll") for (int u = r - 1; u >= 0; u--) {
                    const int s = s0 + u;
                    const int half = gs >> (u + 1);
                    _Pragma("unroll") for (int k1 = 0; k1 < gs; k1++) {
                        if (k1 & half) continue;
                        const int lb = (e0 + k1 * T) >> (LOGP - s);
                        const ulonglong2 w = tw[((bm + seg) << s) + lb];
                        bfly_gs(x[k1], x[k1 + half], w.x, w.y, q, q2);
                    }
                }
            }
        }
        if (rr + 1 < NR) {
            if (rr > 0) __syncthreads();    // everyone has read the previous round's layout
            _Pragma("unroll") for (int qg = 0; qg < ng; qg++)
                _Pragma("unroll") for (int k = 0; k < gs; k++) sm[saddr(elem(qg, k))] = v[qg * gs + k];
        } else {
            // the last pass of a transform leaves canonical residues: forward rows
            // reduce [0, 4q) -> [0, q); inverse columns multiply by 1/N (full
            // reduction).  The first pass leaves its lazy range for the second.
            ulonglong2 ni = make_ulonglong2(0, 0);
            if (scale_out) ni = ninv[pid];
            _Pragma("unroll") for (int qg = 0; qg < ng; qg++)
                _Pragma("unroll") for (int k = 0; k < gs; k++) {
                    u64 y = v[qg * gs + k];
                    if (scale_out)
                        y = shoup_mul(y, ni.x, ni.y, q);
                    else if (!COLS && !INV)
                        y = reduce4(y, q, q2);
                    a[gaddr(elem(qg, k))] = y;
                }
        }
    }
}

template <int LOGP, bool COLS, bool INV>
void launch_pass(Ctx *c, u64 *data, const LimbList &ll, int n_sub, int scale_out)
{
    constexpr int P = 1 << LOGP;
    // sub-transforms per CTA: as many as fit a 4096-word tile, fewer when the
    // batch is small so the grid still covers the SMs (columns keep >= 4
    // consecutive words per row for coalescing)
    int G = std::min(TILE / P, n_sub);
    const int gmin = COLS ? 4 : 1;
    while (G > gmin && (long)(n_sub / G) * ll.n < 2 * 152) G /= 2;
    int logG = 0;
    while ((1 << logG) < G) logG++;
    const int threads = G * P / 8;
    const size_t smem = (size_t)(G * P + (G * P >> 4) + 1) * 8;
    dim3 grid(n_sub / G, ll.n);
    const ulonglong2 *tw = INV ? c->d_tw_inv.as<ulonglong2>() : c->d_tw_fwd.as<ulonglong2>();
    k_ntt_pass<LOGP, COLS, INV><<<grid, threads, smem, c->stream>>>(data, c->logN, logG, ll, tw,
                                                                   c->d_ninv.as<ulonglong2>(),
                                                                   c->d_pinfo.as<PrimeInfo>(), scale_out);
}

template <bool COLS, bool INV>
void dispatch(Ctx *c, int logp, u64 *data, const LimbList &ll, int n_sub, int scale_out)
{
    switch (logp) {
    case 5: launch_pass<5, COLS, INV>(c, data, ll, n_sub, scale_out); break;
    case 6: launch_pass<6, COLS, INV>(c, data, ll, n_sub, scale_out); break;
    case 7: launch_pass<7, COLS, INV>(c, data, ll, n_sub, scale_out); break;
    case 8: launch_pass<8, COLS, INV>(c, data, ll, n_sub, scale_out); break;
    default: fail(HELRM_E_PARAM, "unsupported NTT size");
    }
}

void run(Ctx *c, u64 *data, const std::vector<std::pair<u32, int>> &limbs, bool inverse)
{
    if (limbs.empty()) return;
    const int logN = c->logN, logN1 = logN / 2, logN2 = logN - logN1;
    const int N1 = 1 << logN1, N2 = 1 << logN2;
    KTimer kt(c, "ntt", 16.0 * c->N * limbs.size());   // algorithmic: each limb read and written once
    for (size_t b = 0; b < limbs.size(); b += MAX_LIMBS) {
        LimbList ll;
        ll.n = (int)std::min<size_t>(MAX_LIMBS, limbs.size() - b);
        for (int i = 0; i < ll.n; i++) {
            ll.off[i] = limbs[b + i].first;
            ll.pid[i] = (unsigned short)limbs[b + i].second;
        }
        if (!inverse) {
            dispatch<true, false>(c, logN1, data, ll, N2, 0);
            dispatch<false, false>(c, logN2, data, ll, N1, 0);
        } else {
            dispatch<false, true>(c, logN2, data, ll, N1, 0);
            dispatch<true, true>(c, logN1, data, ll, N2, 1);
        }
        c->launches += 2;
        CUDA_CHECK(cudaGetLastError());
    }
}

}  // namespace

namespace k {

void ntt_list(Ctx *c, u64 *base, const std::vector<std::pair<u32, int>> &limbs, bool inverse)
{
    run(c, base, limbs, inverse);
}

// Contiguous limbs described by a LimbMap; the launch list is built on the
// stack (no heap or device allocation on this path).
static void run_map(Ctx *c, u64 *data, int n_limbs, LimbMap map, bool inverse)
{
    if (n_limbs <= 0) return;
    const int logN = c->logN, logN1 = logN / 2, logN2 = logN - logN1;
    const int N1 = 1 << logN1, N2 = 1 << logN2;
    KTimer kt(c, "ntt", 16.0 * c->N * n_limbs);
    for (int b = 0; b < n_limbs; b += MAX_LIMBS) {
        LimbList ll;
        ll.n = std::min(MAX_LIMBS, n_limbs - b);
        for (int i = 0; i < ll.n; i++) {
            ll.off[i] = (u32)(b + i);
            ll.pid[i] = (unsigned short)map.pid(b + i);
        }
        if (!inverse) {
            dispatch<true, false>(c, logN1, data, ll, N2, 0);
            dispatch<false, false>(c, logN2, data, ll, N1, 0);
        } else {
            dispatch<false, true>(c, logN2, data, ll, N1, 0);
            dispatch<true, true>(c, logN1, data, ll, N2, 1);
        }
        c->launches += 2;
        CUDA_CHECK(cudaGetLastError());
    }
}

void ntt_map_noheap(Ctx *c, u64 *data, int n_limbs, LimbMap map, bool inverse)
{
    run_map(c, data, n_limbs, map, inverse);
}

static std::vector<std::pair<u32, int>> from_map(int n_limbs, LimbMap map)
{
    std::vector<std::pair<u32, int>> v(n_limbs);
    for (int l = 0; l < n_limbs; l++) v[l] = {(u32)l, map.pid(l)};
    return v;
}

void ntt_fwd(Ctx *c, u64 *data, int n_limbs, LimbMap map)
{
    if (n_limbs > 0) run(c, data, from_map(n_limbs, map), false);
}

void ntt_inv(Ctx *c, u64 *data, int n_limbs, LimbMap map)
{
    if (n_limbs > 0) run(c, data, from_map(n_limbs, map), true);
}

}  // namespace k
}  // namespace helrm
