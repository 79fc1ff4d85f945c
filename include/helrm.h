/*
 * helrm.h -- C ABI of the GB300 (sm_103a) encrypted-DLRM library.
 *
 * HE-LRM (Garimella, Ebel, De Micheli, Reagen; arXiv 2506.18150) evaluates a
 * DLRM on CKKS-encrypted inputs: the client digit-decomposes each categorical
 * index, one-hot encodes the digits, packs every table's selectors into one
 * vector and encrypts it (Sec. 4.1, Sec. 4.2.2); the server runs the bottom MLP,
 * the block-diagonally packed embedding lookup y = E^T s and the top MLP, each
 * a plaintext-matrix x ciphertext-vector product evaluated with the
 * double-hoisted baby-step giant-step method (Sec. 2.1.4, Sec. 3.2.1), and
 * returns an encrypted logit (Sec. 5.3).  The CKKS operations are those of the
 * paper's appendix "CKKS operations".
 *
 * Conventions for every call:
 *  - The return value is a helrm_status.  On error the outputs are left
 *    untouched, *out handles are set to NULL, nothing aborts, and the message
 *    is available from helrm_last_error(ctx).
 *  - Handles are opaque and owned by the library; release them with
 *    helrm_free().  Host arrays passed in are read during the call (copied as
 *    needed) and stay owned by the caller.  Pointers named d_* are device
 *    pointers; every other pointer is a host pointer.
 *  - All GPU work is ordered on the context's CUDA stream (the one given to
 *    helrm_ctx_create, e.g. a PyTorch stream).  Calls that return host data
 *    synchronise that stream before returning; the others return once the work
 *    is enqueued.
 *  - Polynomials are stored on the device in RNS form, limb-major
 *    [limb][coefficient], u64 residues in [0, q), in the NTT (evaluation)
 *    domain.  Export/import use the coefficient domain.
 *  - One context per host thread; a context is not thread-safe.
 *
 * Readings of points the paper leaves open (prime choice, noise
 * distributions, PRNG, key-switching gadget, rounding of ModDown and rescale,
 * slot order, layouts and level schedule) are fixed so that the library and
 * an independent CPU oracle compute bit-identical ciphertexts from the same
 * seeds and the same integer plaintexts.  They are listed in the project's
 * design notes.
 */
#ifndef HELRM_H
#define HELRM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HELRM_OK = 0,
    HELRM_E_INVAL = -1,   /* bad argument, size, handle or corrupted input */
    HELRM_E_PARAM = -2,   /* unsupported parameter set */
    HELRM_E_LEVEL = -3,   /* operand level mismatch or no level left */
    HELRM_E_SCALE = -4,   /* operand scale mismatch */
    HELRM_E_NOKEY = -5,   /* missing rotation / relinearisation key */
    HELRM_E_NOMEM = -6,   /* device allocation failed or memory cap reached */
    HELRM_E_CUDA = -7,    /* CUDA runtime error */
    HELRM_E_TIMEOUT = -8  /* a bounded device-side wait ran out */
} helrm_status;

/*
 * CKKS parameters (appendix "CKKS operations": R = Z[X]/(X^N+1), Q = prod q_i).
 *   log_n      N = 2^log_n, 10 <= log_n <= 16; slots n = N/2.
 *   n_q        L+1 ciphertext primes, 1..32;  q_bits[i] their bit sizes (30..60).
 *   n_p        K special primes for key switching, 1..8, each of p_bits (30..60).
 *   alpha      primes per key-switching digit (1..8); dnum = ceil((L+1)/alpha).
 *   log2_scale default scale Delta = 2^log2_scale.
 * Primes: q = 1 mod 2N, for each requested size the largest unused one below
 * 2^bits, q_0..q_L in order, then the special primes.
 */
typedef struct {
    uint32_t log_n;
    uint32_t n_q;
    const uint32_t *q_bits;
    uint32_t n_p;
    uint32_t p_bits;
    uint32_t alpha;
    double log2_scale;
} helrm_params;

typedef struct helrm_ctx helrm_ctx;
typedef struct helrm_sk helrm_sk;       /* secret key (device) */
typedef struct helrm_evk helrm_evk;     /* public, relinearisation and rotation keys (device) */
typedef struct helrm_pt helrm_pt;       /* plaintext polynomial (device) */
typedef struct helrm_ct helrm_ct;       /* ciphertext (device) */
typedef struct helrm_ptmat helrm_ptmat; /* encoded BSGS diagonals of one matrix (device) */
typedef struct helrm_emb helrm_emb;     /* packed embedding tables (device) */
typedef struct helrm_model helrm_model; /* compiled DLRM (device) */
typedef struct helrm_batch helrm_batch; /* a batch of clients for lockstep inference */
typedef struct helrm_server helrm_server; /* request loop with continuous batching */

/* ------------------------------------------------------------------ context */
/* Create a context on `cuda_device`, ordering work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Derives the primes and
 * uploads the NTT and base-conversion tables.  Errors: HELRM_E_PARAM. */
helrm_status helrm_ctx_create(const helrm_params *params, int cuda_device, void *cuda_stream,
                              helrm_ctx **out);
/* primes_out: L+1+K values, q_0..q_L then p_0..p_{K-1}.  psi_out (optional,
 * may be NULL): the primitive 2N-th root used by the NTT for each prime
 * (psi = g^((q-1)/2N), g the smallest quadratic non-residue). */
helrm_status helrm_ctx_primes(const helrm_ctx *ctx, uint64_t *primes_out, uint64_t *psi_out);
/* dims_out[0..5] = N, n (slots), L, K, alpha, dnum at level L. */
helrm_status helrm_ctx_dims(const helrm_ctx *ctx, uint32_t *dims_out);
/* Cap the bytes of device memory the context may hold; 0 = no cap.  An
 * allocation past the cap fails with HELRM_E_NOMEM (admission control). */
helrm_status helrm_ctx_set_memory_cap(helrm_ctx *ctx, uint64_t bytes);
/* Bytes currently held by the context's handles and scratch. */
helrm_status helrm_ctx_memory_in_use(const helrm_ctx *ctx, uint64_t *bytes);
/* Wait for all work enqueued on the context's stream. */
helrm_status helrm_ctx_synchronize(helrm_ctx *ctx);
/* Number of library kernels launched so far on this context. */
helrm_status helrm_ctx_launch_count(const helrm_ctx *ctx, uint64_t *count);
/* Self-test of the device-side timeout path (the paper has no counterpart).
 * Every wait of the library's pipelined kernels on a shared-memory barrier is
 * bounded: when it runs out, the kernel records HELRM_E_TIMEOUT in the
 * context's error word and returns, and the next synchronising call reports
 * it.  This call launches one CTA that waits, for at most `polls` polls
 * (1..2^20), on a barrier that nothing arrives at, and so returns
 * HELRM_E_TIMEOUT with the context still usable afterwards. */
helrm_status helrm_ctx_wait_selftest(helrm_ctx *ctx, uint32_t polls);
/* The NTT launch shapes the context chose when it was created: for limb
 * counts per launch <= 4, <= 16, <= 64 and above (out[3b], out[3b+1],
 * out[3b+2]; out holds 12 words), the words per CTA tile, the CTA count, in
 * multiples of the SM count, below which tiles are split, and the elements
 * per thread (8: radix-8 rounds; 4: radix-4 rounds, N = 2^16 only).
 * Creation times every candidate shape on scratch limbs and keeps the
 * fastest (set HELRM_NTT_AUTOTUNE=0 in the environment to keep the defaults
 * 1024 / 2 / 8, HELRM_NTT_EPT=4 or 8 to try one width only); every shape
 * computes the same result. */
helrm_status helrm_ctx_ntt_tuning(const helrm_ctx *ctx, uint32_t *out);
/* Kernel timing: enable != 0 clears previous records and brackets every
 * library kernel (each NTT counts as one, both passes) with CUDA events on
 * the context stream; 0 stops recording.  Adds a little launch overhead. */
helrm_status helrm_ctx_profile(helrm_ctx *ctx, int enable);
/* Synchronise and summarise the records: one line per kernel,
 * "name launches total_ms algorithmic_bytes\n", into buf (len bytes, always
 * NUL-terminated); *needed (optional) receives the full length + 1. */
helrm_status helrm_ctx_profile_report(helrm_ctx *ctx, char *buf, uint64_t len, uint64_t *needed);
/* The same records one per line in launch order, "name ms algorithmic_bytes\n"
 * (an NTT record's bytes are 16 N per limb, so they give its limb count). */
helrm_status helrm_ctx_profile_records(helrm_ctx *ctx, char *buf, uint64_t len, uint64_t *needed);

/* ------------------------------------------------------------- raw NTT (a2) */
/* In-place negacyclic NTT of n_limbs contiguous limbs of N u64 at d_data;
 * limb l uses prime index first_prime + l (0..L+K, QP order).  Forward: input
 * in [0,q) coefficient order, output ahat[i] = a(psi^(2 brv(i) + 1))
 * (bit-reversed evaluation order); inverse undoes it, including the 1/N.
 * The buffer is owned by the caller. */
helrm_status helrm_ntt(helrm_ctx *ctx, uint64_t *d_data, uint32_t n_limbs, uint32_t first_prime,
                       int inverse);

/* Integer ceiling of the transform (measurement only; the paper has no
 * counterpart): the register-resident rate of the arithmetic the NTT and the
 * inner products run, with no memory traffic, on blocks_per_sm x (SM count)
 * CTAs of 256 threads, each thread repeating `iters` times: kind 0 a radix-8
 * round of 12 lazy forward butterflies, 1 the same for the inverse
 * butterflies, 2 eight 64 x 64 -> 128-bit multiply-accumulates (the
 * library's carry-chained form), 3 eight Shoup modular products, 4 the same
 * sums as 2 from four 32 x 32 -> 64-bit products with explicit carries, 5
 * the same sums for operands below 2^40 as three carry-free 64-bit column
 * sums of 20 x 20-bit products.  *ops_per_s receives butterflies (0, 1),
 * multiply-accumulates (2, 4, 5) or products (3) per second, timed with CUDA
 * events on the context's stream (synchronous).  HELRM_E_INVAL for an
 * unknown kind or blocks_per_sm outside [1, 32]. */
helrm_status helrm_alu_peak(helrm_ctx *ctx, int32_t kind, uint32_t blocks_per_sm, uint32_t iters,
                            double *ops_per_s);

/* ---------------------------------------------------------------- keys (a1) */
/* Key generation from a 64-bit seed (ChaCha20 streams, as for the oracle):
 * ternary secret s, public key (-a s + e, a), the relinearisation key (s^2)
 * and one rotation key per step in rot_steps (slot shifts, negative = right;
 * duplicates and 0 ignored).  Keys are generated over the full QP basis and
 * stay resident on the device. */
helrm_status helrm_keygen(helrm_ctx *ctx, uint64_t seed, const int32_t *rot_steps, uint32_t n_rot,
                          helrm_sk **sk_out, helrm_evk **evk_out);
/* Key generation for one model: the same secret key, public key and key
 * values as helrm_keygen(seed) with the model's rotations, but each rotation
 * key is generated only up to the highest level at which the model uses it,
 * and the relinearisation key up to the highest level of a ciphertext
 * product (a key of level l holds dnum(l) digits over q_0..q_l and the special
 * primes; every value equals the full key's, so ciphertexts are unchanged).
 * Using such a key above its level fails with HELRM_E_NOKEY.  Serving many
 * clients this way needs a fraction of the memory of full keys (the paper
 * reports about 200 MiB per full key, Sec. 2.1.3). */
helrm_status helrm_model_keygen(helrm_ctx *ctx, const helrm_model *m, uint64_t seed, helrm_sk **sk_out,
                                helrm_evk **evk_out);
/* Add rotation keys for more steps to an existing key set. */
helrm_status helrm_evk_add_rotations(helrm_ctx *ctx, const helrm_sk *sk, helrm_evk *evk,
                                     const int32_t *rot_steps, uint32_t n_rot);
/* Total device bytes of the evaluation keys. */
helrm_status helrm_evk_bytes(const helrm_evk *evk, uint64_t *bytes);

/* --------------------------------------------------------- plaintexts (a1) */
/* m = round(scale * sigma^-1(z)) for n_slots real slots z (rest zero), at
 * `level` (limbs q_0..q_level).  slot j is the evaluation at zeta^(5^j). */
helrm_status helrm_encode(helrm_ctx *ctx, const double *slots, uint32_t n_slots, int32_t level,
                          double scale, helrm_pt **out);
/* Plaintext from N signed integer coefficients (|c| < 2^62). */
helrm_status helrm_pt_import(helrm_ctx *ctx, const int64_t *coeffs, int32_t level, double scale,
                             helrm_pt **out);
/* Signed coefficients of a plaintext (centred mod q_0; exact when |c| < q_0/2). */
helrm_status helrm_pt_export(helrm_ctx *ctx, const helrm_pt *pt, int64_t *coeffs_out);

/* ------------------------------------------------------- ciphertexts (a1, a14) */
/* (v*pk_b + e0 + m, v*pk_a + e1) at the plaintext's level; v ternary, e0 and
 * e1 centred binomial, all drawn from `seed`. */
helrm_status helrm_encrypt(helrm_ctx *ctx, const helrm_evk *evk, const helrm_pt *pt, uint64_t seed,
                           helrm_ct **out);
/* Decrypt (m = c0 + c1 s on q_0, centred; requires |m| < q_0/2) and decode
 * the first n_slots slots into slots_out. */
helrm_status helrm_decrypt(helrm_ctx *ctx, const helrm_sk *sk, const helrm_ct *ct, double *slots_out,
                           uint32_t n_slots);
/* Coefficient-domain export: coeffs_out holds 2 x (level+1) x N u64 (c0 limbs
 * then c1 limbs, canonical residues); level/scale optional (may be NULL). */
helrm_status helrm_ct_export(helrm_ctx *ctx, const helrm_ct *ct, uint64_t *coeffs_out, int32_t *level,
                             double *scale);
/* Import the same layout.  A residue >= its prime gives HELRM_E_INVAL. */
helrm_status helrm_ct_import(helrm_ctx *ctx, const uint64_t *coeffs, int32_t level, double scale,
                             helrm_ct **out);
helrm_status helrm_ct_info(const helrm_ct *ct, int32_t *level, double *scale);

/* ----------------------------------------------------- ciphertext ops (a2-a10) */
helrm_status helrm_add(helrm_ctx *ctx, const helrm_ct *a, const helrm_ct *b, helrm_ct **out);
helrm_status helrm_sub(helrm_ctx *ctx, const helrm_ct *a, const helrm_ct *b, helrm_ct **out);
helrm_status helrm_add_pt(helrm_ctx *ctx, const helrm_ct *a, const helrm_pt *pt, helrm_ct **out);
/* Slot-wise product with a plaintext; the scale becomes scale_a * scale_pt
 * (no rescale). */
helrm_status helrm_mul_pt(helrm_ctx *ctx, const helrm_ct *a, const helrm_pt *pt, helrm_ct **out);
/* ct x ct: tensor, relinearise with the s^2 key, rescale (appendix:
 * "Multiplication ... followed by a rescaling procedure"). */
helrm_status helrm_mul(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a, const helrm_ct *b,
                       helrm_ct **out);
/* out = p(x) slot-wise for p(x) = sum_k coeffs[k] x^k, degree d = n_coeffs - 1
 * >= 1 with coeffs[d] != 0 (the polynomial activations of Sec. 2.1.4 /
 * Sec. 5.4).  The needed powers x^k = x^a x^(k-a) (a the largest power of
 * two below k) are ct x ct products; each term a_k x^k is the power at the
 * deepest power's level L_c times the integer round_half_away(a_k s_k),
 * s_k = target_scale q_{L_c} / scale(x^k); the sum is rescaled once and a_0
 * added as the integer round_half_away(a_0 scale) in every slot.  Consumes
 * ceil(log2 d) + 1 levels; the output scale is target_scale up to FP64
 * rounding.  Errors: HELRM_E_LEVEL if the input level is too low,
 * HELRM_E_INVAL for a constant polynomial or a zero leading coefficient. */
helrm_status helrm_poly_eval(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *x, const double *coeffs,
                             uint32_t n_coeffs, double target_scale, helrm_ct **out);
/* Drop q_level: out = round(x / q_level) (centred remainder). */
helrm_status helrm_rescale(helrm_ctx *ctx, const helrm_ct *a, helrm_ct **out);
/* Keep limbs q_0..q_level (level <= current). */
helrm_status helrm_drop_level(helrm_ctx *ctx, const helrm_ct *a, int32_t level, helrm_ct **out);
/* Cyclic left shift of the slots by `step` (appendix "Rotation"):
 * X -> X^(5^step mod 2N) then hybrid key switching (ModUp, key inner
 * product, ModDown).  HELRM_E_NOKEY if the key is missing. */
helrm_status helrm_rotate(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a, int32_t step,
                          helrm_ct **out);
/* n rotations of one ciphertext sharing one ModUp (hoisting); outs[i] for steps[i]. */
helrm_status helrm_rotate_hoisted(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a,
                                  const int32_t *steps, uint32_t n, helrm_ct **outs);

/* ------------------------------------------------------------ matvec (a3-a8) */
/* Encode the BSGS diagonals of the rows x cols row-major FP64 matrix W, padded
 * to out_pad x in_pad (powers of two, <= n): D = min(in_pad, out_pad) extended
 * diagonals diag_i[j] = W[j mod out_pad, (j+i) mod in_pad], split i = g n1 + b
 * (n1 = min(D, max(16, D / 8)) baby steps, n2 = D / n1 giant steps), pre-rotated by -g n1 and
 * encoded over the QP basis at `level` with scale q_level * target_scale /
 * ct_scale.  All-zero diagonals are skipped. */
helrm_status helrm_ptmat_prepare(helrm_ctx *ctx, const double *W, uint32_t rows, uint32_t cols,
                                 uint32_t in_pad, uint32_t out_pad, int32_t level, double ct_scale,
                                 double target_scale, helrm_ptmat **out);
/* info_out[0..5] = D, n1, n2, number of non-zero diagonals, number of fold
 * levels, level. */
helrm_status helrm_ptmat_info(const helrm_ptmat *m, uint32_t *info_out);
/* Rotation steps the matvec needs; steps_out may be NULL to query the count. */
helrm_status helrm_ptmat_rotations(const helrm_ptmat *m, int32_t *steps_out, uint32_t *n_out);
/* Replace the encoded diagonals by `count` plaintexts of N signed
 * coefficients each, in (g, b) order of the non-zero diagonals. */
helrm_status helrm_ptmat_import(helrm_ctx *ctx, helrm_ptmat *m, const int64_t *coeffs, uint32_t count);
/* y = W x: double-hoisted BSGS (one ModUp of c1 shared by the baby steps, the
 * diagonal products accumulated over QP, giant steps rotated in QP, one final
 * ModDown), rescale, then for a wide matrix the folds: the sum of
 * rot(y, j out_pad) over j < in_pad / out_pad, in levels of up to 3 hoisted
 * rotations (strides out_pad, 4 out_pad, 16 out_pad, ...).  The output is
 * W x replicated with period out_pad, one level lower, at target_scale.
 * n_in must be 1. */
helrm_status helrm_ptct_matvec(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ptmat *m,
                               const helrm_ct *in, uint32_t n_in, helrm_ct **out);

/* ------------------------------------------------------- embeddings (a11) */
/* Pack n_tables compressed tables block-diagonally (Sec. 4.2.2): table t with
 * card[t] rows keeps one plain table if card[t] <= threshold (threshold 0
 * means base_p: Sec. 5.2 compresses only the tables above a size threshold),
 * else l_t = ceil(log_p card[t]) digit tables of base_p rows; tables[t] points to
 * its digit tables stacked (sum of rows) x dim, FP32 row-major.  Output rows
 * of table t are [out_offset + dim t, out_offset + dim (t+1)) of a vector of
 * period out_pad; the selector vector (all digits' one-hots concatenated,
 * table by table) has period in_pad = next power of two.  Prepared at
 * `level` for the given scales.  A selector wider than the n slots spans
 * ceil(width / n) ciphertexts (Sec. 5.4: 18 and 85 for the least compressed
 * Criteo models): ciphertext c holds columns [c n, min((c+1) n, width)) with
 * their own period pow2ceil(columns), and each has its own matrix
 * (helrm_emb_matrix); the lookup is the sum of the per-ciphertext products
 * (helrm_embedding_lookup_multi). */
helrm_status helrm_emb_prepare(helrm_ctx *ctx, uint32_t n_tables, const uint64_t *card, uint32_t base_p,
                               uint64_t threshold, uint32_t dim, const float *const *tables,
                               uint32_t out_offset, uint32_t out_pad, int32_t level, double ct_scale,
                               double target_scale, helrm_emb **out);
/* Client packing: little-endian base-p digits of each index, one one-hot per
 * digit, concatenated; slots_out gets n_slots values (selector replicated with
 * its period).  For a selector of C > 1 ciphertexts n_slots must be C x n:
 * block c holds ciphertext c's columns, replicated with their period. */
helrm_status helrm_query_pack(const helrm_emb *emb, const uint64_t *indices, double *slots_out,
                              uint32_t n_slots);
/* Number of ciphertexts the selector spans (1 when it fits n slots). */
helrm_status helrm_emb_chunks(const helrm_emb *emb, uint32_t *n_chunks);
/* The encoded lookup matrix of ciphertext `chunk` (owned by the embedding:
 * valid while it lives, never freed by the caller); use it with
 * helrm_ptmat_info / helrm_ptmat_rotations / helrm_ptmat_import. */
helrm_status helrm_emb_matrix(const helrm_emb *emb, uint32_t chunk, helrm_ptmat **out);
/* Selector width (before padding) and its period. */
helrm_status helrm_emb_info(const helrm_emb *emb, uint32_t *width, uint32_t *period);
/* y = M^T sel for the packed selector ciphertext (n_sel must be 1). */
helrm_status helrm_embedding_lookup(helrm_ctx *ctx, const helrm_evk *evk, const helrm_emb *emb,
                                    const helrm_ct *sel, uint32_t n_sel, helrm_ct **out);
/* The lookup for a selector of n_sel = helrm_emb_chunks ciphertexts:
 * y = sum_c M_c^T sel_c, each term one BSGS matvec (one level), added. */
helrm_status helrm_embedding_lookup_multi(helrm_ctx *ctx, const helrm_evk *evk, const helrm_emb *emb,
                                          const helrm_ct *const *sel, uint32_t n_sel, helrm_ct **out);

/* ------------------------------------------------------------- DLRM (a12-a14) */
typedef struct {
    uint32_t n_dense;
    uint32_t n_bottom;               /* bottom layers; widths[0] = n_dense, last = dim */
    const uint32_t *bottom_widths;   /* n_bottom + 1 */
    const double *const *bottom_W;   /* [layer] -> out x in row-major */
    const double *const *bottom_b;   /* [layer] -> out */
    uint32_t n_top;                  /* top layers; last width 1 */
    const uint32_t *top_widths;      /* n_top + 1; widths[0] = dim + pairs (dot) or dim (T+1) (concat) */
    const double *const *top_W;
    const double *const *top_b;
    uint32_t n_tables;
    const uint64_t *cards;
    uint32_t base_p;
    uint32_t dim;                    /* must be 16 */
    const float *const *tables;      /* as for helrm_emb_prepare */
    int32_t interaction;             /* 0 = pairwise dot, 1 = concatenation */
    uint64_t threshold;              /* tables with more rows are digit-decomposed (0 = base_p) */
    uint32_t act_degree;             /* 0: the activation is x^2; d >= 1: the polynomial below */
    const double *act_coeffs;        /* a_0 .. a_d (powers of x, a_d != 0), see helrm_poly_eval */
    uint32_t boot_bottom;            /* bit i (1 <= i < n_bottom): bootstrap before bottom layer i */
    uint32_t boot_z;                 /* != 0: bootstrap z = h + e (+ ones) before the interaction */
    uint32_t boot_top;               /* bit i (1 <= i < n_top): bootstrap before top layer i */
    const double *boot_coeffs;       /* 17 values: the bootstraps' cosine polynomial (power basis, see
                                        helrm_boot_desc), or NULL: the library's interpolant */
} helrm_model_desc;

/* Compile the model: layouts, as-late-as-possible levels (the logit ends at
 * level 0), all diagonals, biases and masks encoded on the device.  Each
 * activation (after every bottom layer and every top layer but the last)
 * costs one level for x^2, or ceil(log2 d) + 1 for a degree-d polynomial: it
 * is evaluated without a_0 (helrm_poly_eval's schedule), and a_0 is then added
 * as a plaintext on the layer's real outputs only, so that the layout's zero
 * padding stays zero.
 * Bootstrap points (boot_bottom, boot_z, boot_top; the paper's Criteo models
 * with polynomial activations bootstrap between layers, Sec. 5.4) split the
 * network into segments, each planned as late as possible so that it ends at
 * level 0; there a bootstrap (helrm_bootstrap's pipeline with n_s the
 * ciphertext's slot period, K = 24, r = 6, degree 16, 2^8 boost, on the
 * bootstrappable chain: 60-bit primes above the compute levels) lifts the
 * ciphertext, and it is dropped to the first level of the next segment.
 * Every segment must fit in the compute levels (L minus the 13 a bootstrap
 * uses).  The plaintexts of the bootstraps (CoeffToSlot, then SlotToCoeff
 * diagonals per point, in model order) follow the model's in the canonical
 * order.  helrm_model_keygen then draws a sparse secret (h = 192) and adds
 * the bootstraps' rotation keys, the conjugation key and a full-level
 * relinearisation key.
 * Errors: HELRM_E_PARAM if the chain is too short or a layout exceeds n. */
helrm_status helrm_model_create(helrm_ctx *ctx, const helrm_model_desc *desc, helrm_model **out);
/* info_out[0..9] = level of ct_dense, level of ct_sel, level of z, level of
 * the top input, dense period, selector period, W_z, W_u, plaintext count,
 * n_sel (the number of selector ciphertexts a query carries; 1 unless the
 * selector is wider than n slots).  The selector period is that of the
 * first selector ciphertext. */
helrm_status helrm_model_info(const helrm_model *m, uint32_t *info_out);
helrm_status helrm_model_rotations(const helrm_model *m, int32_t *steps_out, uint32_t *n_out);
/* Replace / read all encoded plaintexts (count x N signed coefficients) in
 * the canonical order: per bottom layer its diagonals, its bias, then (a
 * polynomial activation with a_0 != 0) its a_0 plaintext; the embedding
 * diagonals (selector ciphertext by selector ciphertext); (dot) the ones
 * block and masks 0..S; per top layer the same as per bottom layer. */
helrm_status helrm_model_import_plaintexts(helrm_ctx *ctx, helrm_model *m, const int64_t *coeffs,
                                           uint32_t count);
helrm_status helrm_model_export_plaintexts(helrm_ctx *ctx, const helrm_model *m, int64_t *coeffs,
                                           uint32_t count);
/* Client side (a1): pack, encode and encrypt one query: ct_dense with `seed`
 * at its level; ct_sel must hold n_sel (helrm_model_info [9]) handles and
 * receives the selector ciphertexts, ciphertext k encrypted with
 * seed + 1 + k.  dense: n_dense values; indices: one per table. */
helrm_status helrm_encrypt_query(helrm_ctx *ctx, const helrm_evk *evk, const helrm_model *m,
                                 const double *dense, const uint64_t *indices, uint64_t seed,
                                 helrm_ct **ct_dense, helrm_ct **ct_sel);
/* Server side (a2-a13): the encrypted logit (slot 0, level 0).  For a model
 * with n_sel = 1; helrm_infer_multi takes the general case. */
helrm_status helrm_infer(helrm_ctx *ctx, const helrm_evk *evk, const helrm_model *m,
                         const helrm_ct *ct_dense, const helrm_ct *ct_sel, helrm_ct **logit);
/* Server side for a query whose selector spans n_sel ciphertexts (the
 * model's n_sel, else HELRM_E_INVAL): the embedding lookup is the sum of the
 * n_sel per-ciphertext products; the rest is helrm_infer. */
helrm_status helrm_infer_multi(helrm_ctx *ctx, const helrm_evk *evk, const helrm_model *m,
                               const helrm_ct *ct_dense, const helrm_ct *const *ct_sel, uint32_t n_sel,
                               helrm_ct **logit);
/* Client side (a14): decrypt slot 0 and apply the sigmoid. */
helrm_status helrm_decrypt_logit(helrm_ctx *ctx, const helrm_sk *sk, const helrm_ct *logit,
                                 double *logit_out, double *prob_out);
/* The whole protocol for n_queries queries from host buffers: pack, encode,
 * encrypt, infer, decrypt.  dense: n_queries x n_dense; indices: n_queries x
 * n_tables; logits_out / probs_out: n_queries (probs_out may be NULL).
 * Query q is encrypted with seed + (1 + n_sel) q (seed + 2q for n_sel = 1). */
helrm_status helrm_infer_e2e(helrm_ctx *ctx, const helrm_sk *sk, const helrm_evk *evk,
                             const helrm_model *m, const double *dense, const uint64_t *indices,
                             uint32_t n_queries, uint64_t seed, double *logits_out, double *probs_out);

/* The same protocol with every buffer on the device (d_dense: n_queries x
 * n_dense FP64, d_indices: n_queries x n_tables u64, d_logits / d_probs:
 * n_queries FP64, d_probs may be NULL).  Nothing is copied to or from the
 * host and the call does not synchronise.  An index outside its table sets no
 * selector slot for that table (its embedding decrypts to zero); indices are
 * not range-checked on the host. */
helrm_status helrm_infer_e2e_device(helrm_ctx *ctx, const helrm_sk *sk, const helrm_evk *evk,
                                    const helrm_model *m, const double *d_dense, const uint64_t *d_indices,
                                    uint32_t n_queries, uint64_t seed, double *d_logits, double *d_probs);

/* ------------------------------------------------ batched inference (a2-a13) */
/* Lockstep batching of many clients' queries of one model.  Each query goes
 * through exactly the integer operations of helrm_infer, so every logit
 * ciphertext is bit-identical to the one helrm_infer returns for that query
 * alone; the batch only changes the launch shape: every NTT, base
 * conversion, key inner product and elementwise step is one launch for all
 * queries, and the fused baby-step + BSGS kernel reads each weight diagonal
 * once per batch (the diagonals are shared by all clients, Sec. 3.2.1), while
 * each query streams its own client's keys.
 *
 * helrm_batch_create fixes the model and the clients: evks[q] is the
 * evaluation key set of the client of query q (entries may repeat; each needs
 * the model's rotations).  It builds the per-client key tables on the device.
 * The model and the key sets must outlive the batch.  Errors: HELRM_E_NOKEY
 * if a key set lacks a rotation the model needs. */
helrm_status helrm_batch_create(helrm_ctx *ctx, const helrm_model *m, uint32_t n, const helrm_evk *const *evks,
                                helrm_batch **out);
/* enable != 0: run the batch's server path as a CUDA graph.  The first
 * helrm_infer_batch after enabling captures it on buffers the batch owns (one
 * eager run sizes them, then the capture); every call copies its inputs into
 * those buffers, launches the graph and copies the logits out.  The kernels
 * and their order are those of the eager path, so results are identical.
 * Inputs must keep the levels and scales of the captured call.  Must not be
 * combined with helrm_ctx_profile. */
helrm_status helrm_batch_set_graph(helrm_ctx *ctx, helrm_batch *b, int enable);
/* Server side for the n queries of the batch: ct_dense[q] and the n_sel
 * selector ciphertexts ct_sel[q n_sel + k] at the model's levels
 * (helrm_encrypt_query with evks[q]); logits[q] receives the
 * encrypted logit of query q (level 0), as helrm_infer.  Stream ordered, no
 * synchronisation. */
helrm_status helrm_infer_batch(helrm_ctx *ctx, const helrm_batch *b, const helrm_ct *const *ct_dense,
                               const helrm_ct *const *ct_sel, helrm_ct **logits);
/* The whole protocol for the batch from device buffers: query q (d_dense row
 * q, d_indices row q) is packed and encrypted under evks[q] with
 * seed + (1 + n_sel) q,
 * the batch is inferred in lockstep, and logit q is decrypted with sks[q]
 * into d_logits[q].  Nothing is copied to the host; no synchronisation. */
helrm_status helrm_infer_batch_e2e_device(helrm_ctx *ctx, const helrm_batch *b, const helrm_sk *const *sks,
                                         const double *d_dense, const uint64_t *d_indices, uint64_t seed,
                                         double *d_logits);
/* The same protocol for the batch from host buffers (dense: n x n_dense FP64,
 * indices: n x n_tables u64, logits_out: n FP64): the inputs are copied to
 * the device, the batch runs as helrm_infer_batch_e2e_device (as a CUDA graph
 * when enabled), the logits are copied back, and the call synchronises.  As
 * with the device variant, an index outside its table sets no selector slot. */
helrm_status helrm_infer_batch_e2e(helrm_ctx *ctx, const helrm_batch *b, const helrm_sk *const *sks,
                                   const double *dense, const uint64_t *indices, uint64_t seed,
                                   double *logits_out);

/* --------------------------------------------------- serving (a2-a13, batched) */
/* A request loop over lockstep batches.  Clients register their model and
 * evaluation keys once; the keys stay resident on the device.  The server
 * has n_slots batch slots, each its own CUDA stream: batches on different
 * slots run concurrently on the GPU.  A batch holds up to max_batch requests
 * of one model (a batch of one runs helrm_infer itself, so n_slots = 1,
 * max_batch = 1 is the plain one-request-at-a-time path).  mem_budget bounds
 * the device bytes that in-flight batches may hold (0 = unbounded); a
 * context memory cap (helrm_ctx_set_memory_cap), when set, takes precedence.
 * Errors: HELRM_E_INVAL for sizes outside 1..16 slots, 1..256 per batch. */
helrm_status helrm_server_create(helrm_ctx *ctx, uint32_t n_slots, uint32_t max_batch, uint64_t mem_budget,
                                 helrm_server **out);
/* Register a client: the model its queries use and its evaluation keys
 * (both must outlive the server).  *client_id receives its index.  Any model
 * is accepted, including one whose selector spans several ciphertexts. */
helrm_status helrm_server_add_client(helrm_ctx *ctx, helrm_server *s, const helrm_model *m, const helrm_evk *evk,
                                     uint32_t *client_id);
typedef struct {
    double p50_ms, p99_ms, mean_ms, max_ms;  /* request latency: completion - arrival */
    double makespan_s;                        /* first arrival to last completion */
    double throughput;                        /* requests / makespan_s */
    uint32_t n_batches, max_batch, max_inflight;
    double mean_batch;
} helrm_serve_stats;
/* Replay n timed requests through the loop.  Request r arrives at
 * arrival_s[r] seconds (sorted ascending) from client[r] with its query
 * ciphertexts (helrm_encrypt_query, already on the device): ct_dense[r], and
 * in ct_sel the n_sel selector ciphertexts of the client's model (one unless
 * the selector is wider than the slots), request after request, so ct_sel
 * holds the sum of the requests' n_sel.  Each pass of
 * the loop admits the requests that have arrived, launches a batch on every
 * free slot that the memory budget allows (oldest pending request first,
 * with more pending requests of the same model), and polls the slots for
 * completion.  Requests arriving while others run start as soon as a slot
 * and memory free up, overlapping on the device.  When nothing is pending or
 * running, the loop skips ahead to the next arrival.  logits_out[r] receives
 * request r's encrypted logit (bit-identical to helrm_infer's);
 * latency_ms_out[r] its latency; stats (optional) the summary.  On error all
 * logits handed out are released and set to NULL. */
helrm_status helrm_server_run(helrm_ctx *ctx, helrm_server *s, uint32_t n, const double *arrival_s,
                              const uint32_t *client, const helrm_ct *const *ct_dense, const helrm_ct *const *ct_sel,
                              helrm_ct **logits_out, double *latency_ms_out, helrm_serve_stats *stats);

/* ------------------------------------------------- allocation-free rescale */
/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: a host whose GPU memory is owned by another
 * allocator (for example a framework's caching pool that has reserved the
 * device), a real-time serving loop that must not take the implicit
 * synchronisation of an allocation, or code that may only touch buffers it
 * was handed.  It computes what helrm_rescale computes and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   d_in    device, n_polys x (level+1) x N u64, NTT domain (the layout of the
 *           library's ciphertexts: c0 limbs then c1 limbs for n_polys = 2);
 *   d_out   device, n_polys x level x N u64, NTT domain; must not overlap d_in
 *           (HELRM_E_INVAL if it does).
 * Its one scratch buffer is a static device array of 2 x 65536 u64 words
 * (1 MiB); n_polys x N above that limit is rejected with HELRM_E_INVAL.
 * helrm_ctx_create does the set-up, where allocating is allowed: it looks up
 * the array's device address (cudaGetSymbolAddress) and loads its module and
 * kernels, so every GPU on which a context is created holds the array from
 * then until the process exits, and this call itself loads nothing.  All
 * calls share the array and it keeps the last call's contents (each call
 * overwrites what it reads): calls that overlap on the GPU (different streams
 * or contexts on the same device) race on it.  Work is ordered on the
 * context's stream; the call does not synchronise.  Errors: HELRM_E_INVAL
 * (NULL, overlapping or oversized buffers), HELRM_E_LEVEL (level outside
 * [1, L]), HELRM_E_CUDA (a failed launch or copy). */
helrm_status helrm_rescale_noalloc(helrm_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int32_t level,
                                   uint32_t n_polys);

/* ----------------------------------------------------- bootstrapping (Sec. 2.1.4) */
/* The paper refreshes levels by bootstrapping (Sec. 2.1.4; 12 or 5 bootstraps
 * in its Criteo models, Sec. 5.4) without giving the steps; the library runs
 * the standard pipeline for a ciphertext whose real slots are periodic with
 * period n_s (2 n_s <= N/2):
 *   boost (x 2^log2_boost at level 0), ModRaise (the level-0 residues,
 *   centred, as residues of q_0..q_L), SubSum (ct += rot(ct, n_s 2^i) up to
 *   N/2: the trace onto X^(N/(2 n_s))), CoeffToSlot (a BSGS product C of
 *   U^H / (2 n_s), U[i][k] = exp(i pi (5^i k mod 4 n_s) / (2 n_s)) the
 *   n_s x 2 n_s slot matrix, then C + conj(C): the slots, period 2 n_s,
 *   hold the coefficients over q_0 and 2^r), EvalMod (minus 1/(4 2^r), an even polynomial fit of cos(2 pi y) on
 *   |y| <= (K + 1/2)/2^r, r double angles 2c^2 - 1: sin(2 pi u)) and
 *   SlotToCoeff (U times q_0 / (2 pi 2^log2_boost s_ref), one fold).
 * It consumes cts_levels + depth(degree) + r + 1 levels from the top
 * (depth as for helrm_poly_eval).  Precision needs EvalMod at about 2^60:
 * the bootstrappable chain puts 60-bit primes at the top (cts_levels = 1,
 * eval_scale = 2^60); on an all-40-bit chain (cts_levels = 2, eval_scale =
 * 2^40) about 4 bits of a unit message survive.  The keys must come from a
 * sparse secret (helrm_keygen_ex, h about 192 for K = 24) with the rotations
 * of helrm_boot_rotations and the conjugation key. */
typedef struct helrm_boot helrm_boot;
typedef struct {
    uint32_t n_s;          /* slot period (power of two, 2 n_s <= N/2) */
    uint32_t K;            /* |I| the sine covers (about 6 sqrt(h/12)) */
    uint32_t r;            /* double angles */
    uint32_t degree;       /* even degree of the cosine fit */
    uint32_t log2_boost;   /* the message is multiplied by 2^log2_boost at level 0 */
    uint32_t cts_levels;   /* 1 or 2 rescales after CoeffToSlot */
    double s_ref;          /* input scale the SlotToCoeff constant assumes */
    double eval_scale;     /* scale EvalMod runs at */
    const double *coeffs;  /* degree + 1 power-basis coefficients in y, or NULL: the library's
                              interpolant at the degree + 1 Chebyshev points of the interval */
} helrm_boot_desc;
/* Encodes the two matrices (CoeffToSlot at level L, SlotToCoeff at the level
 * EvalMod ends on) on the device.  HELRM_E_PARAM if the chain is
 * too short, HELRM_E_INVAL for other bad parameters. */
helrm_status helrm_boot_create(helrm_ctx *ctx, const helrm_boot_desc *desc, helrm_boot **out);
/* info_out[6]: n_s, top level, SlotToCoeff level, output level, number of
 * encoded diagonals (CoeffToSlot's, then SlotToCoeff's), degree. */
helrm_status helrm_boot_info(const helrm_boot *b, uint32_t *info_out);
/* The slot rotations the keys must cover (SubSum, the BSGS steps, the fold). */
helrm_status helrm_boot_rotations(const helrm_boot *b, int32_t *steps_out, uint32_t *n_out);
/* The cosine polynomial in use (degree + 1 values). */
helrm_status helrm_boot_coeffs(const helrm_boot *b, double *coeffs_out, uint32_t n);
/* Borrowed matrix handles (0: CoeffToSlot, 1: SlotToCoeff), valid while b
 * lives; for helrm_ptmat_import / helrm_ptmat_export. */
helrm_status helrm_boot_matrix(const helrm_boot *b, uint32_t which, helrm_ptmat **out);
/* out = the refreshed ciphertext at the output level, scale about Delta
 * (times in->scale / s_ref), slots decoding to the input's.  The input may
 * be at any level (it is dropped to level 0); it is not modified.  stages
 * (optional, NULL or 5 entries) receives copies of the intermediate
 * ciphertexts: after ModRaise, SubSum, CoeffToSlot, EvalMod, and the output;
 * the caller frees them.  HELRM_E_NOKEY without the rotation or conjugation
 * keys. */
helrm_status helrm_bootstrap(helrm_ctx *ctx, const helrm_evk *evk, const helrm_boot *b, const helrm_ct *in,
                             helrm_ct **out, helrm_ct **stages);
/* helrm_keygen with a choice of secret: hamming_weight = 0 is the dense
 * ternary secret of helrm_keygen (the same keys); h > 0 gives exactly h
 * coefficients in {-1, +1} (ChaCha20 stream words 0..N-1 rank the positions,
 * the h smallest (word, position) pairs are non-zero, bit 0 of word N + i is
 * the sign of position i).  conj != 0 adds the key of X -> X^(2N-1). */
helrm_status helrm_keygen_ex(helrm_ctx *ctx, uint64_t seed, uint32_t hamming_weight, const int32_t *rot_steps,
                             uint32_t n_rot, int conj, helrm_sk **sk_out, helrm_evk **evk_out);
/* X -> X^(2N-1) with the key switch: every slot conjugated. */
helrm_status helrm_conjugate(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a, helrm_ct **out);
/* The diagonals of a prepared matrix as centred coefficients (limb 0,
 * count x N int64, the order of helrm_ptmat_import). */
helrm_status helrm_ptmat_export(helrm_ctx *ctx, const helrm_ptmat *m, int64_t *coeffs, uint32_t count);

/* --------------------------------------------------------------- misc */
/* Release any handle (context last; handles must not outlive their context). */
void helrm_free(void *handle);
const char *helrm_last_error(const helrm_ctx *ctx);
const char *helrm_status_string(helrm_status s);

#ifdef __cplusplus
}
#endif
#endif /* HELRM_H */
