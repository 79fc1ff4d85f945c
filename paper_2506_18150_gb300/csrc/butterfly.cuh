// butterfly.cuh -- the lazy Harvey butterflies of the 64-bit NTT (ntt.cu),
// shared with the register-resident measurement of their throughput
// (peak.cu), so that both run the same code.
//
// Twiddles carry Shoup quotients; values stay in [0, 4q) forward and [0, 2q)
// inverse (q < 2^62) and are corrected once at the end of a transform.
#pragma once

#include "core.cuh"

namespace helrm {

// Shoup product without its final correction: a * w mod q in [0, 2q).
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q) { return a * w - mulhi64(a, wp) * q; }
// x >= m ? x - m : x, as one 64-bit min (x - m wraps above x when x < m)
__device__ __forceinline__ u64 csub(u64 x, u64 m)
{
    const u64 y = x - m;
    return y < x ? y : x;
}
// forward (Cooley-Tukey): x0, x1 in [0, 4q) -> [0, 4q)
__device__ __forceinline__ void bfly_ct(u64 &x0, u64 &x1, u64 w, u64 wp, u64 q, u64 q2)
{
    const u64 a = csub(x0, q2);
    const u64 t = shoup_lazy(x1, w, wp, q);
    x0 = a + t;
    x1 = a - t + q2;
}
// inverse (Gentleman-Sande): x0, x1 in [0, 2q) -> [0, 2q)
__device__ __forceinline__ void bfly_gs(u64 &x0, u64 &x1, u64 w, u64 wp, u64 q, u64 q2)
{
    const u64 s = csub(x0 + x1, q2);
    const u64 t = x0 - x1 + q2;
    x0 = s;
    x1 = shoup_lazy(t, w, wp, q);
}

}  // namespace helrm
