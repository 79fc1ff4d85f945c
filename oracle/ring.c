/*
 * oracle/ring.c -- TEST INFRASTRUCTURE, not part of the library.
 *
 * Plain CPU reference arithmetic for the RNS polynomial ring
 * R_q = Z_q[X]/(X^N + 1) used by CKKS (HE-LRM appendix "CKKS operations":
 * ciphertexts live in R_Q^2 with Q a product of word-sized primes, and every
 * operation is limb-wise modular arithmetic).  Only tests/, the package smoke
 * check and the bench's CPU-baseline leg may load this file's shared object.
 *
 * Every modular product is the definition itself: a 128-bit product reduced
 * with the C `%` operator.  There is no Montgomery, Barrett or Shoup trick, no
 * lazy reduction and no blocking, so each line can be checked by eye.
 *
 * Two independent ways to multiply in R_q are provided:
 *   - the schoolbook negacyclic convolution, O(N^2), straight from
 *     X^N = -1 (the "exact" reference used to pin everything else);
 *   - a textbook radix-2 NTT (bit-reversal copy, then iterative
 *     Cooley-Tukey over a cyclic length-N transform with the 2N-th root psi
 *     folded in as a pre-twist), O(N log N).
 * Arrays of several limbs are [limb][coefficient], limb-major; loops over
 * limbs are OpenMP-parallel, which changes no result.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

static u64 mul_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * (u128)b) % q); }
static u64 add_mod(u64 a, u64 b, u64 q) { return (u64)((((u128)a) + b) % q); }
static u64 sub_mod(u64 a, u64 b, u64 q)
{
    a %= q;
    b %= q;
    return a >= b ? a - b : q - (b - a);
}
static u64 pow_mod(u64 b, u64 e, u64 q)
{
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mul_mod(r, b, q);
        b = mul_mod(b, b, q);
        e >>= 1;
    }
    return r;
}
/* q is prime, so a^(q-2) is the inverse (Fermat). */
static u64 inv_mod(u64 a, u64 q) { return pow_mod(a, q - 2, q); }

u64 orc_mul_mod(u64 a, u64 b, u64 q) { return mul_mod(a, b, q); }
u64 orc_pow_mod(u64 b, u64 e, u64 q) { return pow_mod(b, e, q); }

/* out[k] = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j  (mod q): X^N = -1. */
void orc_negacyclic_schoolbook(const u64 *a, const u64 *b, u64 *out, u64 n, u64 q)
{
    for (u64 k = 0; k < n; k++) {
        u64 pos = 0, neg = 0;
        for (u64 i = 0; i <= k; i++) pos = add_mod(pos, mul_mod(a[i], b[k - i], q), q);
        for (u64 i = k + 1; i < n; i++) neg = add_mod(neg, mul_mod(a[i], b[n + k - i], q), q);
        out[k] = sub_mod(pos, neg, q);
    }
}

static void bit_reverse_copy(u64 *a, u64 n)
{
    for (u64 i = 1, j = 0; i < n; i++) {
        u64 bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            u64 t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
}

/* Cyclic DFT over Z_q: A_k = sum_i a_i w^(ik), w a primitive n-th root. */
static void cyclic_ntt(u64 *a, u64 n, u64 q, u64 w)
{
    bit_reverse_copy(a, n);
    for (u64 len = 2; len <= n; len <<= 1) {
        u64 wl = pow_mod(w, n / len, q);
        for (u64 s = 0; s < n; s += len) {
            u64 x = 1;
            for (u64 j = 0; j < len / 2; j++) {
                u64 u = a[s + j];
                u64 v = mul_mod(a[s + j + len / 2], x, q);
                a[s + j] = add_mod(u, v, q);
                a[s + j + len / 2] = sub_mod(u, v, q);
                x = mul_mod(x, wl, q);
            }
        }
    }
}

/*
 * Negacyclic transform: forward gives ahat[k] = a(psi^(2k+1)) in natural
 * order (pre-twist by psi^i, then the cyclic transform with w = psi^2);
 * inverse undoes it exactly.  psi must be a primitive 2N-th root mod q.
 */
static void negacyclic_ntt(u64 *a, u64 n, u64 q, u64 psi, int inverse)
{
    if (!inverse) {
        u64 t = 1;
        for (u64 i = 0; i < n; i++) {
            a[i] = mul_mod(a[i], t, q);
            t = mul_mod(t, psi, q);
        }
        cyclic_ntt(a, n, q, mul_mod(psi, psi, q));
    } else {
        u64 psi_inv = inv_mod(psi, q);
        cyclic_ntt(a, n, q, mul_mod(psi_inv, psi_inv, q));
        u64 t = inv_mod(n % q, q);
        for (u64 i = 0; i < n; i++) {
            a[i] = mul_mod(a[i], t, q);
            t = mul_mod(t, psi_inv, q);
        }
    }
}

void orc_ntt_batch(u64 *a, u64 n, u64 limbs, const u64 *q, const u64 *psi, int inverse)
{
#pragma omp parallel for schedule(dynamic)
    for (u64 l = 0; l < limbs; l++) negacyclic_ntt(a + l * n, n, q[l], psi[l], inverse);
}

/* out = a * b in R_q, limb by limb, through the textbook NTT. */
void orc_polymul_batch(const u64 *a, const u64 *b, u64 *out, u64 n, u64 limbs, const u64 *q,
                       const u64 *psi)
{
#pragma omp parallel for schedule(dynamic)
    for (u64 l = 0; l < limbs; l++) {
        u64 *ta = (u64 *)malloc(n * sizeof(u64));
        u64 *tb = (u64 *)malloc(n * sizeof(u64));
        memcpy(ta, a + l * n, n * sizeof(u64));
        memcpy(tb, b + l * n, n * sizeof(u64));
        negacyclic_ntt(ta, n, q[l], psi[l], 0);
        negacyclic_ntt(tb, n, q[l], psi[l], 0);
        for (u64 i = 0; i < n; i++) ta[i] = mul_mod(ta[i], tb[i], q[l]);
        negacyclic_ntt(ta, n, q[l], psi[l], 1);
        memcpy(out + l * n, ta, n * sizeof(u64));
        free(ta);
        free(tb);
    }
}

/* out = a * b (pointwise, mod q of the limb). */
void orc_mul_batch(const u64 *a, const u64 *b, u64 *out, u64 n, u64 limbs, const u64 *q)
{
#pragma omp parallel for schedule(static)
    for (u64 l = 0; l < limbs; l++)
        for (u64 i = 0; i < n; i++) out[l * n + i] = mul_mod(a[l * n + i], b[l * n + i], q[l]);
}

/* out = a * c_l (one scalar per limb). Inputs may exceed q; the result is < q. */
void orc_mul_scalar_batch(const u64 *a, const u64 *c, u64 *out, u64 n, u64 limbs, const u64 *q)
{
#pragma omp parallel for schedule(static)
    for (u64 l = 0; l < limbs; l++)
        for (u64 i = 0; i < n; i++) out[l * n + i] = mul_mod(a[l * n + i], c[l], q[l]);
}

/* out = (hi * 2^64 + lo) mod q_l: a 128-bit integer reduced by the definition. */
void orc_reduce128_batch(const u64 *hi, const u64 *lo, u64 *out, u64 n, u64 limbs, const u64 *q)
{
#pragma omp parallel for schedule(static)
    for (u64 l = 0; l < limbs; l++)
        for (u64 i = 0; i < n; i++) {
            u128 v = ((u128)hi[l * n + i] << 64) | lo[l * n + i];
            out[l * n + i] = (u64)(v % q[l]);
        }
}
