// api.cu -- extern "C" entry points declared in include/helrm.h.
//
// Every entry point validates its handles, converts C++ errors and CUDA
// errors into a helrm_status, records the message on the context, and leaves
// its outputs untouched (out handles NULL) on failure.
#include <cstring>
#include <new>

#include "model.cuh"

namespace helrm {
Ciphertext *ct_poly_eval(Ctx *c, const EvalKey *evk, const Ciphertext *x, const std::vector<double> &a,
                         double target);
Ctx *ctx_create(const helrm_params *p, int device, void *stream);
struct Emb;
struct Model;
Emb *emb_prepare(Ctx *c, const std::vector<u64> &cards, int base, u64 threshold, int dim, const float *const *tables,
                 int out_offset, int out_pad, int level, double ct_scale, double target_scale);
void emb_pack_host(const Emb *e, const u64 *indices, std::vector<double> &sel);
const PtMatrix *emb_matrix_of(const Emb *e);
int emb_n_chunks(const Emb *e);
PtMatrix *emb_chunk(const Emb *e, int c);
int emb_chunk_period(const Emb *e, int c);
Ciphertext *emb_lookup_multi(Ctx *c, const EvalKey *evk, const Emb *e, const std::vector<const Ciphertext *> &sel);
void emb_info(const Emb *e, u32 *width, u32 *period);
Ctx *emb_ctx(const Emb *e);
Model *model_create(Ctx *c, const helrm_model_desc *d);
void model_import(Ctx *c, Model *m, const i64 *coeffs, u32 count);
void model_export(Ctx *c, Model *m, i64 *coeffs, u32 count);
Ciphertext *model_infer(Ctx *c, const EvalKey *evk, const Model *m, const Ciphertext *ct_dense,
                        const std::vector<const Ciphertext *> &ct_sel);
void model_encrypt_query(Ctx *c, const EvalKey *evk, const Model *m, const double *dense, const u64 *indices,
                         u64 seed, Ciphertext **ct_dense, std::vector<Ciphertext *> &ct_sel, bool on_device);
int model_n_sel(const Model *m);
void model_info(const Model *m, u32 *o);
std::vector<int> model_rotations(const Model *m);
std::vector<std::pair<int, int>> model_key_levels(const Model *m, int *relin_level);
Ctx *model_ctx(const Model *m);
u32 model_n_dense(const Model *m);
u32 model_n_tables(const Model *m);
struct Batch;
Batch *batch_create(Ctx *c, const Model *m, const std::vector<const EvalKey *> &evk);
std::vector<Ciphertext *> model_infer_batch(Ctx *c, const Batch *bt, const std::vector<const Ciphertext *> &ct_dense,
                                            const std::vector<const Ciphertext *> &ct_sel);
size_t batch_size(const Batch *b);
const Model *batch_model(const Batch *b);
const EvalKey *batch_evk(const Batch *b, size_t q);
std::vector<Ciphertext *> model_infer_batch_graph(Ctx *c, Batch *bt, const std::vector<const Ciphertext *> &ct_dense,
                                                  const std::vector<const Ciphertext *> &ct_sel);
void batch_set_graph(Batch *b, bool on);
bool batch_uses_graph(const Batch *b);
struct Server;
Server *server_create(Ctx *c, int n_slots, int max_batch, u64 budget);
u32 server_add_client(Server *s, const Model *m, const EvalKey *evk);
u32 server_sel_count(const Server *s, u32 n, const u32 *client);
void server_run(Server *s, u32 n, const double *arrival, const u32 *client, const Ciphertext *const *ct_dense,
                const Ciphertext *const *ct_sel, Ciphertext **out, double *latency_ms, helrm_serve_stats *st);
}  // namespace helrm

using namespace helrm;

namespace {

template <class T>
T *as(const void *h, u32 kind, const char *what)
{
    HCHECK(h, HELRM_E_INVAL, std::string(what) + " is NULL");
    const Handle *hh = (const Handle *)h;
    HCHECK(hh->kind == kind, HELRM_E_INVAL, std::string(what) + " is not a valid handle of its type");
    return (T *)h;
}
Ctx *C(const helrm_ctx *c) { return as<Ctx>(c, KIND_CTX, "ctx"); }
const SecretKey *SK(const helrm_sk *s) { return as<SecretKey>(s, KIND_SK, "secret key"); }
EvalKey *EVK(const helrm_evk *e) { return as<EvalKey>(e, KIND_EVK, "evaluation key"); }
Plaintext *PT(const helrm_pt *p) { return as<Plaintext>(p, KIND_PT, "plaintext"); }
Ciphertext *CT(const helrm_ct *p) { return as<Ciphertext>(p, KIND_CT, "ciphertext"); }
PtMatrix *PM(const helrm_ptmat *p) { return as<PtMatrix>(p, KIND_PTMAT, "ptmat"); }
Emb *EMB(const helrm_emb *p) { return as<Emb>(p, KIND_EMB, "embedding"); }
Model *MOD(const helrm_model *p) { return as<Model>(p, KIND_MODEL, "model"); }
Batch *BAT(const helrm_batch *p) { return as<Batch>(p, KIND_BATCH, "batch"); }
Server *SRV(const helrm_server *p) { return as<Server>(p, KIND_SERVER, "server"); }
Boot *BT(const helrm_boot *p) { return as<Boot>(p, KIND_BOOT, "bootstrapping"); }

Ctx *ctx_or_null(const void *h)
{
    if (!h) return nullptr;
    const Handle *hh = (const Handle *)h;
    return hh->kind == KIND_CTX ? (Ctx *)h : nullptr;
}


template <class T>
void set_out(T **out, T *v)
{
    *out = v;
}

}  // namespace

extern "C" {

// ------------------------------------------------------------------ context
helrm_status helrm_ctx_create(const helrm_params *params, int cuda_device, void *cuda_stream, helrm_ctx **out)
{
    if (out) *out = nullptr;
    return guard(nullptr, [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        *out = (helrm_ctx *)ctx_create(params, cuda_device, cuda_stream);
    });
}

helrm_status helrm_ctx_primes(const helrm_ctx *ctx, uint64_t *primes_out, uint64_t *psi_out)
{
    Ctx *c = ctx_or_null(ctx);
    return guard(c, [&] {
        Ctx *cc = C(ctx);
        HCHECK(primes_out, HELRM_E_INVAL, "primes_out is NULL");
        std::memcpy(primes_out, cc->primes.data(), cc->primes.size() * 8);
        if (psi_out) std::memcpy(psi_out, cc->psi.data(), cc->psi.size() * 8);
    });
}

helrm_status helrm_ctx_dims(const helrm_ctx *ctx, uint32_t *d)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(d, HELRM_E_INVAL, "dims_out is NULL");
        d[0] = c->N;
        d[1] = c->n_slots;
        d[2] = c->L;
        d[3] = c->K;
        d[4] = c->alpha;
        d[5] = c->dnum(c->L);
    });
}

helrm_status helrm_ctx_set_memory_cap(helrm_ctx *ctx, uint64_t bytes)
{
    return guard(ctx_or_null(ctx), [&] { C(ctx)->mem_cap = bytes; });
}

helrm_status helrm_ctx_memory_in_use(const helrm_ctx *ctx, uint64_t *bytes)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(bytes, HELRM_E_INVAL, "bytes is NULL");
        *bytes = C(ctx)->mem_in_use;
    });
}

helrm_status helrm_ctx_synchronize(helrm_ctx *ctx)
{
    return guard(ctx_or_null(ctx), [&] { C(ctx)->check_device_errors(); });
}

helrm_status helrm_ctx_launch_count(const helrm_ctx *ctx, uint64_t *count)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(count, HELRM_E_INVAL, "count is NULL");
        *count = C(ctx)->launches;
    });
}

helrm_status helrm_ctx_wait_selftest(helrm_ctx *ctx, uint32_t polls)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(polls >= 1 && polls <= (1u << 20), HELRM_E_INVAL, "polls must be in [1, 2^20]");
        k::wait_probe(c, (long)polls);
        c->check_device_errors();   // raises HELRM_E_TIMEOUT and clears the word
    });
}

helrm_status helrm_ctx_ntt_tuning(const helrm_ctx *ctx, uint32_t *out)
{
    return guard(ctx_or_null(ctx), [&] {
        const Ctx *c = C(ctx);
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        for (int b = 0; b < 4; b++) {
            out[3 * b] = (uint32_t)c->ntt_tune[b].tile;
            out[3 * b + 1] = (uint32_t)c->ntt_tune[b].mult;
            out[3 * b + 2] = (uint32_t)c->ntt_tune[b].ept;
        }
    });
}

helrm_status helrm_ctx_profile(helrm_ctx *ctx, int enable)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        if (enable) {
            CUDA_CHECK(cudaStreamSynchronize(c->stream));
            for (auto &r : c->prof) {
                c->event_pool.push_back(r.start);
                c->event_pool.push_back(r.stop);
            }
            c->prof.clear();
        }
        c->prof_on = enable != 0;
    });
}

helrm_status helrm_ctx_profile_records(helrm_ctx *ctx, char *buf, uint64_t len, uint64_t *needed)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        std::string s;
        char line[256];
        for (auto &r : c->prof) {
            float ms = 0;
            CUDA_CHECK(cudaEventElapsedTime(&ms, r.start, r.stop));
            snprintf(line, sizeof line, "%s %.6f %.0f\n", r.name, ms, r.bytes);
            s += line;
        }
        if (needed) *needed = s.size() + 1;
        if (buf && len) {
            size_t n = std::min<size_t>(len - 1, s.size());
            std::memcpy(buf, s.data(), n);
            buf[n] = 0;
        }
    });
}

helrm_status helrm_ctx_profile_report(helrm_ctx *ctx, char *buf, uint64_t len, uint64_t *needed)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        struct Agg {
            u64 n = 0;
            double ms = 0, bytes = 0;
        };
        std::map<std::string, Agg> agg;
        for (auto &r : c->prof) {
            float ms = 0;
            CUDA_CHECK(cudaEventElapsedTime(&ms, r.start, r.stop));
            Agg &a = agg[r.name];
            a.n++;
            a.ms += ms;
            a.bytes += r.bytes;
        }
        std::string s;
        char line[256];
        for (auto &kv : agg) {
            snprintf(line, sizeof line, "%s %llu %.6f %.0f\n", kv.first.c_str(), (unsigned long long)kv.second.n,
                     kv.second.ms, kv.second.bytes);
            s += line;
        }
        if (needed) *needed = s.size() + 1;
        if (buf && len) {
            size_t n = std::min<size_t>(len - 1, s.size());
            std::memcpy(buf, s.data(), n);
            buf[n] = 0;
        }
    });
}

helrm_status helrm_alu_peak(helrm_ctx *ctx, int32_t kind, uint32_t blocks_per_sm, uint32_t iters,
                            double *ops_per_s)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(ops_per_s, HELRM_E_INVAL, "ops_per_s is NULL");
        *ops_per_s = k::alu_peak(c, kind, (int)blocks_per_sm, (int)iters);
    });
}

helrm_status helrm_ntt(helrm_ctx *ctx, uint64_t *d_data, uint32_t n_limbs, uint32_t first_prime, int inverse)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(d_data || n_limbs == 0, HELRM_E_INVAL, "d_data is NULL");
        HCHECK((int)first_prime + (int)n_limbs <= c->nP(), HELRM_E_INVAL, "prime index out of range");
        LimbMap m{(int)first_prime, 1 << 30, c->L + 1, 0};
        if (inverse)
            k::ntt_inv(c, d_data, (int)n_limbs, m);
        else
            k::ntt_fwd(c, d_data, (int)n_limbs, m);
    });
}

// ------------------------------------------------------------------ keys
helrm_status helrm_keygen(helrm_ctx *ctx, uint64_t seed, const int32_t *rot_steps, uint32_t n_rot,
                          helrm_sk **sk_out, helrm_evk **evk_out)
{
    if (sk_out) *sk_out = nullptr;
    if (evk_out) *evk_out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(sk_out && evk_out, HELRM_E_INVAL, "output pointers are NULL");
        HCHECK(rot_steps || n_rot == 0, HELRM_E_INVAL, "rot_steps is NULL");
        std::unique_ptr<SecretKey> sk(keygen_sk(c, seed));
        std::unique_ptr<EvalKey> evk(keygen_evk(c, sk.get(), seed));
        keygen_rot(c, sk.get(), evk.get(), std::vector<int>(rot_steps, rot_steps + n_rot));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        *sk_out = (helrm_sk *)sk.release();
        *evk_out = (helrm_evk *)evk.release();
    });
}

helrm_status helrm_model_keygen(helrm_ctx *ctx, const helrm_model *m, uint64_t seed, helrm_sk **sk_out,
                                helrm_evk **evk_out)
{
    if (sk_out) *sk_out = nullptr;
    if (evk_out) *evk_out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(sk_out && evk_out, HELRM_E_INVAL, "output pointers are NULL");
        int rl = 0;
        std::vector<std::pair<int, int>> kl = model_key_levels(MOD(m), &rl);
        std::vector<int> steps, levels;
        for (auto &x : kl) {
            steps.push_back(x.first);
            levels.push_back(x.second);
        }
        // a model with bootstraps needs a sparse secret (the sine covers |I| <= 24)
        const bool boots = MOD(m)->has_boot();
        std::unique_ptr<SecretKey> sk(keygen_sk(c, seed, boots ? 192 : 0));
        std::unique_ptr<EvalKey> evk(keygen_evk(c, sk.get(), seed, rl));
        keygen_rot(c, sk.get(), evk.get(), steps, levels);
        if (boots) keygen_galois(c, sk.get(), evk.get(), {2ull * c->N - 1});
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        *sk_out = (helrm_sk *)sk.release();
        *evk_out = (helrm_evk *)evk.release();
    });
}

helrm_status helrm_evk_add_rotations(helrm_ctx *ctx, const helrm_sk *sk, helrm_evk *evk, const int32_t *rot_steps,
                                     uint32_t n_rot)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(rot_steps || n_rot == 0, HELRM_E_INVAL, "rot_steps is NULL");
        keygen_rot(c, SK(sk), EVK(evk), std::vector<int>(rot_steps, rot_steps + n_rot));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
    });
}

helrm_status helrm_evk_bytes(const helrm_evk *evk, uint64_t *bytes)
{
    return guard(nullptr, [&] {
        EvalKey *e = EVK(evk);
        HCHECK(bytes, HELRM_E_INVAL, "bytes is NULL");
        u64 b = e->pk.bytes + (e->relin ? e->relin->data.bytes : 0);
        for (auto &kv : e->rot) b += kv.second->data.bytes;
        *bytes = b;
    });
}

// ------------------------------------------------------------------ plaintexts
helrm_status helrm_encode(helrm_ctx *ctx, const double *slots, uint32_t n_slots, int32_t level, double scale,
                          helrm_pt **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(out && (slots || n_slots == 0), HELRM_E_INVAL, "NULL argument");
        HCHECK(n_slots <= (u32)c->n_slots, HELRM_E_INVAL, "more values than slots");
        std::unique_ptr<Plaintext> pt(pt_encode(c, slots, (int)n_slots, c->n_slots, level, false, scale, PT_PLAIN));
        c->check_device_errors();
        *out = (helrm_pt *)pt.release();
    });
}

helrm_status helrm_pt_import(helrm_ctx *ctx, const int64_t *coeffs, int32_t level, double scale, helrm_pt **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(out && coeffs, HELRM_E_INVAL, "NULL argument");
        *out = (helrm_pt *)pt_from_signed(c, coeffs, level, false, scale, PT_PLAIN);
    });
}

helrm_status helrm_pt_export(helrm_ctx *ctx, const helrm_pt *pt, int64_t *coeffs_out)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(coeffs_out, HELRM_E_INVAL, "coeffs_out is NULL");
        pt_export_signed(C(ctx), PT(pt), coeffs_out);
    });
}

// ------------------------------------------------------------------ ciphertexts
helrm_status helrm_encrypt(helrm_ctx *ctx, const helrm_evk *evk, const helrm_pt *pt, uint64_t seed, helrm_ct **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        *out = (helrm_ct *)encrypt_pt(C(ctx), EVK(evk), PT(pt), seed);
    });
}

helrm_status helrm_decrypt(helrm_ctx *ctx, const helrm_sk *sk, const helrm_ct *ct, double *slots_out,
                           uint32_t n_slots)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(slots_out || n_slots == 0, HELRM_E_INVAL, "slots_out is NULL");
        decrypt_slots(C(ctx), SK(sk), CT(ct), slots_out, (int)n_slots);
    });
}

helrm_status helrm_ct_export(helrm_ctx *ctx, const helrm_ct *ct, uint64_t *coeffs_out, int32_t *level,
                             double *scale)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        Ciphertext *a = CT(ct);
        HCHECK(coeffs_out, HELRM_E_INVAL, "coeffs_out is NULL");
        const int nq = a->level + 1;
        DevMem t(c, (size_t)2 * nq * c->N * 8);
        k::copy(c, t.u(), a->data.u(), (size_t)2 * nq * c->N);
        k::ntt_inv(c, t.u(), 2 * nq, c->qmap(a->level, 0, nq));
        CUDA_CHECK(cudaMemcpyAsync(coeffs_out, t.ptr, t.bytes, cudaMemcpyDeviceToHost, c->stream));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        if (level) *level = a->level;
        if (scale) *scale = a->scale;
    });
}

helrm_status helrm_ct_import(helrm_ctx *ctx, const uint64_t *coeffs, int32_t level, double scale, helrm_ct **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(out && coeffs, HELRM_E_INVAL, "NULL argument");
        HCHECK(level >= 0 && level <= c->L, HELRM_E_LEVEL, "level out of range");
        const int nq = level + 1;
        std::unique_ptr<Ciphertext> a(new_ct(c, level, scale));
        CUDA_CHECK(cudaMemcpyAsync(a->data.ptr, coeffs, a->data.bytes, cudaMemcpyHostToDevice, c->stream));
        DevMem flag(c, 8);
        CUDA_CHECK(cudaMemsetAsync(flag.ptr, 0, 8, c->stream));
        k::check_range(c, a->data.u(), 2 * nq, c->qmap(level, 0, nq), flag.as<int>());
        int h = 0;
        CUDA_CHECK(cudaMemcpyAsync(&h, flag.ptr, 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        HCHECK(!h, HELRM_E_INVAL, "imported ciphertext has a residue >= its prime");
        k::ntt_fwd(c, a->data.u(), 2 * nq, c->qmap(level, 0, nq));
        *out = (helrm_ct *)a.release();
    });
}

helrm_status helrm_ct_info(const helrm_ct *ct, int32_t *level, double *scale)
{
    return guard(nullptr, [&] {
        Ciphertext *a = CT(ct);
        if (level) *level = a->level;
        if (scale) *scale = a->scale;
    });
}

// ------------------------------------------------------------------ ops
#define CT_OP(body)                                       \
    if (out) *out = nullptr;                              \
    return guard(ctx_or_null(ctx), [&] {                  \
        HCHECK(out, HELRM_E_INVAL, "out is NULL");        \
        Ctx *c = C(ctx);                                  \
        *out = (helrm_ct *)(body);                        \
    })

helrm_status helrm_add(helrm_ctx *ctx, const helrm_ct *a, const helrm_ct *b, helrm_ct **out)
{
    CT_OP(ct_add(c, CT(a), CT(b), false));
}
helrm_status helrm_sub(helrm_ctx *ctx, const helrm_ct *a, const helrm_ct *b, helrm_ct **out)
{
    CT_OP(ct_add(c, CT(a), CT(b), true));
}
helrm_status helrm_add_pt(helrm_ctx *ctx, const helrm_ct *a, const helrm_pt *pt, helrm_ct **out)
{
    CT_OP(ct_add_pt(c, CT(a), PT(pt)));
}
helrm_status helrm_mul_pt(helrm_ctx *ctx, const helrm_ct *a, const helrm_pt *pt, helrm_ct **out)
{
    CT_OP(ct_mul_pt(c, CT(a), PT(pt)));
}
helrm_status helrm_mul(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a, const helrm_ct *b, helrm_ct **out)
{
    CT_OP(ct_mul(c, EVK(evk), CT(a), CT(b)));
}
helrm_status helrm_rescale(helrm_ctx *ctx, const helrm_ct *a, helrm_ct **out) { CT_OP(ct_rescale(c, CT(a))); }
helrm_status helrm_poly_eval(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *x, const double *coeffs,
                             uint32_t n_coeffs, double target_scale, helrm_ct **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out && coeffs, HELRM_E_INVAL, "NULL argument");
        *out = (helrm_ct *)ct_poly_eval(C(ctx), EVK(evk), CT(x), std::vector<double>(coeffs, coeffs + n_coeffs),
                                        target_scale);
    });
}
helrm_status helrm_drop_level(helrm_ctx *ctx, const helrm_ct *a, int32_t level, helrm_ct **out)
{
    CT_OP(ct_drop(c, CT(a), level));
}
helrm_status helrm_rotate(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a, int32_t step, helrm_ct **out)
{
    CT_OP(ct_rotate(c, EVK(evk), CT(a), step));
}

helrm_status helrm_rotate_hoisted(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a, const int32_t *steps,
                                  uint32_t n, helrm_ct **outs)
{
    if (outs)
        for (u32 i = 0; i < n; i++) outs[i] = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(outs && (steps || n == 0), HELRM_E_INVAL, "NULL argument");
        std::vector<Ciphertext *> r;
        ct_rotate_hoisted(c, EVK(evk), CT(a), std::vector<int>(steps, steps + n), r);
        for (u32 i = 0; i < n; i++) outs[i] = (helrm_ct *)r[i];
    });
}

// ------------------------------------------------------------------ matvec
helrm_status helrm_ptmat_prepare(helrm_ctx *ctx, const double *W, uint32_t rows, uint32_t cols, uint32_t in_pad,
                                 uint32_t out_pad, int32_t level, double ct_scale, double target_scale,
                                 helrm_ptmat **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        *out = (helrm_ptmat *)ptmat_prepare(C(ctx), W, (int)rows, (int)cols, (int)in_pad, (int)out_pad, level,
                                            ct_scale, target_scale);
    });
}

helrm_status helrm_ptmat_info(const helrm_ptmat *m, uint32_t *o)
{
    return guard(nullptr, [&] {
        PtMatrix *p = PM(m);
        HCHECK(o, HELRM_E_INVAL, "info_out is NULL");
        o[0] = p->D;
        o[1] = p->n1;
        o[2] = p->n2;
        o[3] = (u32)p->gb.size();
        o[4] = (u32)p->folds.size();
        o[5] = p->level;
    });
}

static void copy_steps(const std::vector<int> &st, int32_t *steps_out, uint32_t *n_out)
{
    HCHECK(n_out, HELRM_E_INVAL, "n_out is NULL");
    if (steps_out) {
        HCHECK(*n_out >= st.size(), HELRM_E_INVAL, "steps_out too small");
        for (size_t i = 0; i < st.size(); i++) steps_out[i] = st[i];
    }
    *n_out = (u32)st.size();
}

helrm_status helrm_ptmat_rotations(const helrm_ptmat *m, int32_t *steps_out, uint32_t *n_out)
{
    return guard(nullptr, [&] { copy_steps(PM(m)->rotations(), steps_out, n_out); });
}

helrm_status helrm_ptmat_import(helrm_ctx *ctx, helrm_ptmat *m, const int64_t *coeffs, uint32_t count)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        PtMatrix *p = PM(m);
        HCHECK(coeffs, HELRM_E_INVAL, "coeffs is NULL");
        HCHECK(count == p->pts.size(), HELRM_E_INVAL, "diagonal count mismatch");
        for (u32 i = 0; i < count; i++)
            p->pts[i].reset(pt_from_signed(c, coeffs + (size_t)i * c->N, p->level, true, p->pt_scale, PT_MONT));
        p->upload_index();
    });
}

helrm_status helrm_ptct_matvec(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ptmat *m, const helrm_ct *in,
                               uint32_t n_in, helrm_ct **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        HCHECK(n_in == 1, HELRM_E_INVAL, "n_in must be 1");
        *out = (helrm_ct *)matvec(C(ctx), EVK(evk), PM(m), CT(in));
    });
}

// ------------------------------------------------------------------ embeddings
helrm_status helrm_emb_prepare(helrm_ctx *ctx, uint32_t n_tables, const uint64_t *card, uint32_t base_p,
                               uint64_t threshold, uint32_t dim, const float *const *tables, uint32_t out_offset,
                               uint32_t out_pad, int32_t level, double ct_scale, double target_scale, helrm_emb **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out && card && n_tables, HELRM_E_INVAL, "NULL argument");
        *out = (helrm_emb *)emb_prepare(C(ctx), std::vector<u64>(card, card + n_tables), (int)base_p, threshold,
                                        (int)dim,
                                        tables, (int)out_offset, (int)out_pad, level, ct_scale, target_scale);
    });
}

helrm_status helrm_query_pack(const helrm_emb *emb, const uint64_t *indices, double *slots_out, uint32_t n_slots)
{
    Ctx *c = nullptr;
    if (emb && ((const Handle *)emb)->kind == KIND_EMB) c = emb_ctx((const Emb *)emb);
    return guard(c, [&] {
        Emb *e = EMB(emb);
        HCHECK(indices && (slots_out || n_slots == 0), HELRM_E_INVAL, "NULL argument");
        std::vector<double> sel;
        emb_pack_host(e, indices, sel);
        u32 w, per;
        emb_info(e, &w, &per);
        const int nc = emb_n_chunks(e);
        if (nc == 1) {
            for (u32 j = 0; j < n_slots; j++) slots_out[j] = (j % per) < w ? sel[j % per] : 0.0;
            return;
        }
        // one block of n slots per ciphertext: chunk c's columns replicated with its period
        const u32 n = (u32)emb_chunk_period(e, 0);
        HCHECK(n_slots == (u32)nc * n, HELRM_E_INVAL, "a multi-ciphertext selector needs n_chunks x n slots");
        for (int k = 0; k < nc; k++) {
            const u32 c0 = (u32)k * n, cw = std::min(n, w - c0), cp = (u32)emb_chunk_period(e, k);
            for (u32 j = 0; j < n; j++) slots_out[(size_t)k * n + j] = (j % cp) < cw ? sel[c0 + j % cp] : 0.0;
        }
    });
}

helrm_status helrm_emb_chunks(const helrm_emb *emb, uint32_t *n_chunks)
{
    return guard(nullptr, [&] {
        HCHECK(n_chunks, HELRM_E_INVAL, "NULL argument");
        *n_chunks = (uint32_t)emb_n_chunks(EMB(emb));
    });
}

helrm_status helrm_emb_matrix(const helrm_emb *emb, uint32_t chunk, helrm_ptmat **out)
{
    return guard(nullptr, [&] {
        const Emb *e = EMB(emb);
        HCHECK(out && chunk < (uint32_t)emb_n_chunks(e), HELRM_E_INVAL, "chunk out of range");
        *out = (helrm_ptmat *)emb_chunk(e, (int)chunk);
    });
}

helrm_status helrm_embedding_lookup_multi(helrm_ctx *ctx, const helrm_evk *evk, const helrm_emb *emb,
                                          const helrm_ct *const *sel, uint32_t n_sel, helrm_ct **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out && sel, HELRM_E_INVAL, "NULL argument");
        std::vector<const Ciphertext *> v;
        for (u32 k = 0; k < n_sel; k++) v.push_back(CT(sel[k]));
        *out = (helrm_ct *)emb_lookup_multi(C(ctx), EVK(evk), EMB(emb), v);
    });
}

helrm_status helrm_emb_info(const helrm_emb *emb, uint32_t *width, uint32_t *period)
{
    return guard(nullptr, [&] {
        HCHECK(width && period, HELRM_E_INVAL, "NULL argument");
        emb_info(EMB(emb), width, period);
    });
}

helrm_status helrm_embedding_lookup(helrm_ctx *ctx, const helrm_evk *evk, const helrm_emb *emb, const helrm_ct *sel,
                                    uint32_t n_sel, helrm_ct **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        HCHECK(n_sel == 1, HELRM_E_INVAL, "n_sel must be 1");
        HCHECK(emb_n_chunks(EMB(emb)) == 1, HELRM_E_INVAL,
               "the selector spans several ciphertexts: use helrm_embedding_lookup_multi");
        *out = (helrm_ct *)matvec(C(ctx), EVK(evk), emb_matrix_of(EMB(emb)), CT(sel));
    });
}

// ------------------------------------------------------------------ model
helrm_status helrm_model_create(helrm_ctx *ctx, const helrm_model_desc *desc, helrm_model **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out && desc, HELRM_E_INVAL, "NULL argument");
        *out = (helrm_model *)model_create(C(ctx), desc);
    });
}

helrm_status helrm_model_info(const helrm_model *m, uint32_t *info_out)
{
    return guard(nullptr, [&] {
        HCHECK(info_out, HELRM_E_INVAL, "info_out is NULL");
        model_info(MOD(m), info_out);
    });
}

helrm_status helrm_model_rotations(const helrm_model *m, int32_t *steps_out, uint32_t *n_out)
{
    return guard(nullptr, [&] { copy_steps(model_rotations(MOD(m)), steps_out, n_out); });
}

helrm_status helrm_model_import_plaintexts(helrm_ctx *ctx, helrm_model *m, const int64_t *coeffs, uint32_t count)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(coeffs, HELRM_E_INVAL, "coeffs is NULL");
        model_import(C(ctx), MOD(m), coeffs, count);
    });
}

helrm_status helrm_model_export_plaintexts(helrm_ctx *ctx, const helrm_model *m, int64_t *coeffs, uint32_t count)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(coeffs, HELRM_E_INVAL, "coeffs is NULL");
        model_export(C(ctx), MOD(m), coeffs, count);
    });
}

helrm_status helrm_encrypt_query(helrm_ctx *ctx, const helrm_evk *evk, const helrm_model *m, const double *dense,
                                 const uint64_t *indices, uint64_t seed, helrm_ct **ct_dense, helrm_ct **ct_sel)
{
    const int ns = (m && ((const Handle *)m)->kind == KIND_MODEL) ? model_n_sel((const Model *)m) : 1;
    if (ct_dense) *ct_dense = nullptr;
    if (ct_sel)
        for (int k2 = 0; k2 < ns; k2++) ct_sel[k2] = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(dense && indices && ct_dense && ct_sel, HELRM_E_INVAL, "NULL argument");
        Ciphertext *a;
        std::vector<Ciphertext *> b;
        model_encrypt_query(C(ctx), EVK(evk), MOD(m), dense, indices, seed, &a, b, false);
        *ct_dense = (helrm_ct *)a;
        for (size_t k2 = 0; k2 < b.size(); k2++) ct_sel[k2] = (helrm_ct *)b[k2];
    });
}

helrm_status helrm_infer(helrm_ctx *ctx, const helrm_evk *evk, const helrm_model *m, const helrm_ct *ct_dense,
                         const helrm_ct *ct_sel, helrm_ct **logit)
{
    return helrm_infer_multi(ctx, evk, m, ct_dense, &ct_sel, 1, logit);
}

helrm_status helrm_infer_multi(helrm_ctx *ctx, const helrm_evk *evk, const helrm_model *m, const helrm_ct *ct_dense,
                               const helrm_ct *const *ct_sel, uint32_t n_sel, helrm_ct **logit)
{
    if (logit) *logit = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(logit && ct_sel, HELRM_E_INVAL, "NULL argument");
        std::vector<const Ciphertext *> s;
        for (u32 k2 = 0; k2 < n_sel; k2++) s.push_back(CT(ct_sel[k2]));
        *logit = (helrm_ct *)model_infer(C(ctx), EVK(evk), MOD(m), CT(ct_dense), s);
    });
}

namespace {
// one query's client side + server side + decryption; query q of a run uses
// the seeds seed + (1 + n_sel) q ... (a fresh seed per ciphertext)
struct QueryCts {
    std::unique_ptr<Ciphertext> dense;
    std::vector<std::unique_ptr<Ciphertext>> sel;
    std::vector<const Ciphertext *> sel_ptrs() const
    {
        std::vector<const Ciphertext *> v;
        for (auto &p : sel) v.push_back(p.get());
        return v;
    }
};
QueryCts encrypt_one(Ctx *c, const EvalKey *evk, const Model *m, const double *dense, const u64 *indices, u64 seed,
                     bool on_device)
{
    Ciphertext *a;
    std::vector<Ciphertext *> b;
    model_encrypt_query(c, evk, m, dense, indices, seed, &a, b, on_device);
    QueryCts r;
    r.dense.reset(a);
    for (auto *p : b) r.sel.emplace_back(p);
    return r;
}
}  // namespace

helrm_status helrm_decrypt_logit(helrm_ctx *ctx, const helrm_sk *sk, const helrm_ct *logit, double *logit_out,
                                 double *prob_out)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(logit_out, HELRM_E_INVAL, "logit_out is NULL");
        double v = 0;
        decrypt_slots(C(ctx), SK(sk), CT(logit), &v, 1);
        *logit_out = v;
        if (prob_out) *prob_out = 1.0 / (1.0 + std::exp(-v));
    });
}

helrm_status helrm_infer_e2e(helrm_ctx *ctx, const helrm_sk *sk, const helrm_evk *evk, const helrm_model *m,
                             const double *dense, const uint64_t *indices, uint32_t n_queries, uint64_t seed,
                             double *logits_out, double *probs_out)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        Model *mm = MOD(m);
        HCHECK((dense && indices && logits_out) || n_queries == 0, HELRM_E_INVAL, "NULL argument");
        const size_t nd = model_n_dense(mm), nt = model_n_tables(mm);
        const u64 stride = 1 + (u64)model_n_sel(mm);
        for (u32 q = 0; q < n_queries; q++) {
            QueryCts x = encrypt_one(c, EVK(evk), mm, dense + q * nd, indices + q * nt, seed + stride * q, false);
            std::unique_ptr<Ciphertext> y(model_infer(c, EVK(evk), mm, x.dense.get(), x.sel_ptrs()));
            double v = 0;
            decrypt_slots(c, SK(sk), y.get(), &v, 1);
            logits_out[q] = v;
            if (probs_out) probs_out[q] = 1.0 / (1.0 + std::exp(-v));
        }
    });
}

helrm_status helrm_infer_e2e_device(helrm_ctx *ctx, const helrm_sk *sk, const helrm_evk *evk, const helrm_model *m,
                                    const double *d_dense, const uint64_t *d_indices, uint32_t n_queries, uint64_t seed,
                                    double *d_logits, double *d_probs)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        Model *mm = MOD(m);
        HCHECK((d_dense && d_indices && d_logits) || n_queries == 0, HELRM_E_INVAL, "NULL argument");
        const size_t nd = model_n_dense(mm), nt = model_n_tables(mm);
        const u64 stride = 1 + (u64)model_n_sel(mm);
        for (u32 q = 0; q < n_queries; q++) {
            QueryCts x = encrypt_one(c, EVK(evk), mm, d_dense + q * nd, d_indices + q * nt, seed + stride * q, true);
            std::unique_ptr<Ciphertext> y(model_infer(c, EVK(evk), mm, x.dense.get(), x.sel_ptrs()));
            decrypt_slots_device(c, SK(sk), y.get(), d_logits + q, 1);
        }
        if (d_probs && n_queries) k::sigmoid(c, d_probs, d_logits, (int)n_queries);
    });
}

// ------------------------------------------------------ batched inference
helrm_status helrm_batch_create(helrm_ctx *ctx, const helrm_model *m, uint32_t n, const helrm_evk *const *evks,
                                helrm_batch **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out && evks && n >= 1, HELRM_E_INVAL, "NULL argument or empty batch");
        std::vector<const EvalKey *> ev;
        for (u32 q = 0; q < n; q++) ev.push_back(EVK(evks[q]));
        *out = (helrm_batch *)batch_create(C(ctx), MOD(m), ev);
    });
}

helrm_status helrm_batch_set_graph(helrm_ctx *ctx, helrm_batch *b, int enable)
{
    return guard(ctx_or_null(ctx), [&] {
        C(ctx);
        batch_set_graph(BAT(b), enable != 0);
    });
}

helrm_status helrm_infer_batch(helrm_ctx *ctx, const helrm_batch *b, const helrm_ct *const *ct_dense,
                               const helrm_ct *const *ct_sel, helrm_ct **logits)
{
    const size_t n = (b && ((const Handle *)b)->kind == KIND_BATCH) ? batch_size((const Batch *)b) : 0;
    if (logits)
        for (size_t q = 0; q < n; q++) logits[q] = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Batch *bt = BAT(b);
        HCHECK(ct_dense && ct_sel && logits, HELRM_E_INVAL, "NULL argument");
        const size_t ns = (size_t)model_n_sel(batch_model(bt));
        std::vector<const Ciphertext *> d, s;
        for (size_t q = 0; q < n; q++) d.push_back(CT(ct_dense[q]));
        for (size_t r = 0; r < n * ns; r++) s.push_back(CT(ct_sel[r]));
        std::vector<Ciphertext *> y = batch_uses_graph(bt) ? model_infer_batch_graph(C(ctx), bt, d, s)
                                                           : model_infer_batch(C(ctx), bt, d, s);
        for (size_t q = 0; q < n; q++) logits[q] = (helrm_ct *)y[q];
    });
}

namespace {
void batch_e2e_device(Ctx *c, Batch *bt, const helrm_sk *const *sks, const double *d_dense, const uint64_t *d_indices,
                      uint64_t seed, double *d_logits);
}

helrm_status helrm_infer_batch_e2e(helrm_ctx *ctx, const helrm_batch *b, const helrm_sk *const *sks,
                                   const double *dense, const uint64_t *indices, uint64_t seed, double *logits_out)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        Batch *bt = BAT(b);
        HCHECK(sks && dense && indices && logits_out, HELRM_E_INVAL, "NULL argument");
        const Model *mm = batch_model(bt);
        const size_t n = batch_size(bt), nd = model_n_dense((Model *)mm), nt = model_n_tables((Model *)mm);
        DevMem dd(c, n * nd * 8), di(c, n * nt * 8), dl(c, n * 8);
        CUDA_CHECK(cudaMemcpyAsync(dd.ptr, dense, n * nd * 8, cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(di.ptr, indices, n * nt * 8, cudaMemcpyHostToDevice, c->stream));
        batch_e2e_device(c, bt, sks, dd.as<double>(), di.u(), seed, dl.as<double>());
        CUDA_CHECK(cudaMemcpyAsync(logits_out, dl.ptr, n * 8, cudaMemcpyDeviceToHost, c->stream));
        c->check_device_errors();
    });
}

helrm_status helrm_infer_batch_e2e_device(helrm_ctx *ctx, const helrm_batch *b, const helrm_sk *const *sks,
                                         const double *d_dense, const uint64_t *d_indices, uint64_t seed,
                                         double *d_logits)
{
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(sks && d_dense && d_indices && d_logits, HELRM_E_INVAL, "NULL argument");
        batch_e2e_device(C(ctx), BAT(b), sks, d_dense, d_indices, seed, d_logits);
    });
}

namespace {
void batch_e2e_device(Ctx *c, Batch *bt, const helrm_sk *const *sks, const double *d_dense, const uint64_t *d_indices,
                      uint64_t seed, double *d_logits)
{
    {
        const Model *mm = batch_model(bt);
        const size_t n = batch_size(bt), nd = model_n_dense((Model *)mm), nt = model_n_tables((Model *)mm);
        std::vector<const SecretKey *> sk;
        for (size_t q = 0; q < n; q++) sk.push_back(SK(sks[q]));
        const u64 stride = 1 + (u64)model_n_sel(mm);
        std::vector<QueryCts> qc;
        std::vector<const Ciphertext *> ad, sd;
        for (size_t q = 0; q < n; q++) {   // client side: each client packs and encrypts its own query
            qc.push_back(encrypt_one(c, batch_evk(bt, q), mm, d_dense + q * nd, d_indices + q * nt, seed + stride * q,
                                     true));
            ad.push_back(qc.back().dense.get());
            for (auto *p : qc.back().sel_ptrs()) sd.push_back(p);
        }
        std::vector<Ciphertext *> y = batch_uses_graph(bt) ? model_infer_batch_graph(c, bt, ad, sd)
                                                           : model_infer_batch(c, bt, ad, sd);
        std::vector<std::unique_ptr<Ciphertext>> yo;
        for (auto *p : y) yo.emplace_back(p);
        for (size_t q = 0; q < n; q++) decrypt_slots_device(c, sk[q], yo[q].get(), d_logits + q, 1);
    }
}
}  // namespace

// ------------------------------------------------------------------ serving
helrm_status helrm_server_create(helrm_ctx *ctx, uint32_t n_slots, uint32_t max_batch, uint64_t mem_budget,
                                 helrm_server **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        *out = (helrm_server *)server_create(C(ctx), (int)n_slots, (int)max_batch, mem_budget);
    });
}

helrm_status helrm_server_add_client(helrm_ctx *ctx, helrm_server *s, const helrm_model *m, const helrm_evk *evk,
                                     uint32_t *client_id)
{
    return guard(ctx_or_null(ctx), [&] {
        C(ctx);
        const u32 id = server_add_client(SRV(s), MOD(m), EVK(evk));
        if (client_id) *client_id = id;
    });
}

helrm_status helrm_server_run(helrm_ctx *ctx, helrm_server *s, uint32_t n, const double *arrival_s,
                              const uint32_t *client, const helrm_ct *const *ct_dense, const helrm_ct *const *ct_sel,
                              helrm_ct **logits_out, double *latency_ms_out, helrm_serve_stats *stats)
{
    if (logits_out)
        for (u32 r = 0; r < n; r++) logits_out[r] = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        C(ctx);
        HCHECK(arrival_s && client && ct_dense && ct_sel && logits_out && latency_ms_out, HELRM_E_INVAL,
               "NULL argument");
        const u32 n_sel = server_sel_count(SRV(s), n, client);
        std::vector<const Ciphertext *> d(n), sl(n_sel);
        for (u32 r = 0; r < n; r++) d[r] = CT(ct_dense[r]);
        for (u32 k = 0; k < n_sel; k++) sl[k] = CT(ct_sel[k]);
        server_run(SRV(s), n, arrival_s, client, d.data(), sl.data(), (Ciphertext **)logits_out, latency_ms_out,
                   stats);
    });
}

// ------------------------------------------------------------------ misc
helrm_status helrm_keygen_ex(helrm_ctx *ctx, uint64_t seed, uint32_t hamming_weight, const int32_t *rot_steps,
                             uint32_t n_rot, int conj, helrm_sk **sk_out, helrm_evk **evk_out)
{
    if (sk_out) *sk_out = nullptr;
    if (evk_out) *evk_out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(sk_out && evk_out, HELRM_E_INVAL, "output pointers are NULL");
        HCHECK(rot_steps || n_rot == 0, HELRM_E_INVAL, "rot_steps is NULL");
        HCHECK(hamming_weight <= (u32)c->N, HELRM_E_INVAL, "hamming_weight above N");
        std::unique_ptr<SecretKey> sk(keygen_sk(c, seed, (int)hamming_weight));
        std::unique_ptr<EvalKey> evk(keygen_evk(c, sk.get(), seed));
        keygen_rot(c, sk.get(), evk.get(), std::vector<int>(rot_steps, rot_steps + n_rot));
        if (conj) keygen_galois(c, sk.get(), evk.get(), {2ull * c->N - 1});
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        *sk_out = (helrm_sk *)sk.release();
        *evk_out = (helrm_evk *)evk.release();
    });
}

helrm_status helrm_conjugate(helrm_ctx *ctx, const helrm_evk *evk, const helrm_ct *a, helrm_ct **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        *out = (helrm_ct *)ct_apply_galois(C(ctx), EVK(evk), CT(a), 2ull * C(ctx)->N - 1);
    });
}

helrm_status helrm_ptmat_export(helrm_ctx *ctx, const helrm_ptmat *m, int64_t *coeffs, uint32_t count)
{
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        const PtMatrix *p = PM(m);
        HCHECK(coeffs, HELRM_E_INVAL, "coeffs is NULL");
        HCHECK(count == p->pts.size(), HELRM_E_INVAL, "diagonal count mismatch");
        for (u32 i = 0; i < count; i++) pt_export_signed(c, p->pts[i].get(), coeffs + (size_t)i * c->N);
    });
}

helrm_status helrm_boot_create(helrm_ctx *ctx, const helrm_boot_desc *desc, helrm_boot **out)
{
    if (out) *out = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        Ctx *c = C(ctx);
        HCHECK(desc && out, HELRM_E_INVAL, "NULL argument");
        BootDesc d{(int)desc->n_s, (int)desc->K, (int)desc->r, (int)desc->degree, (int)desc->log2_boost,
                   (int)desc->cts_levels, desc->s_ref, desc->eval_scale, {}};
        if (desc->coeffs) d.coeffs.assign(desc->coeffs, desc->coeffs + desc->degree + 1);
        std::unique_ptr<Boot> b(boot_create(c, d));
        c->check_device_errors();
        *out = (helrm_boot *)b.release();
    });
}

helrm_status helrm_boot_info(const helrm_boot *bh, uint32_t *info_out)
{
    return guard(nullptr, [&] {
        const Boot *b = BT(bh);
        HCHECK(info_out, HELRM_E_INVAL, "info_out is NULL");
        size_t nd = 0;
        for (PtMatrix *m : b->matrices()) nd += m->pts.size();
        info_out[0] = (u32)b->n_s;
        info_out[1] = (u32)b->level_top;
        info_out[2] = (u32)b->level_stc;
        info_out[3] = (u32)b->level_out;
        info_out[4] = (u32)nd;
        info_out[5] = (u32)b->degree;
    });
}

helrm_status helrm_boot_rotations(const helrm_boot *b, int32_t *steps_out, uint32_t *n_out)
{
    return guard(nullptr, [&] { copy_steps(BT(b)->rotations(), steps_out, n_out); });
}

helrm_status helrm_boot_coeffs(const helrm_boot *bh, double *coeffs_out, uint32_t n)
{
    return guard(nullptr, [&] {
        const Boot *b = BT(bh);
        HCHECK(coeffs_out && n == b->coeffs.size(), HELRM_E_INVAL, "coeffs_out must hold degree + 1 values");
        for (u32 i = 0; i < n; i++) coeffs_out[i] = b->coeffs[i];
    });
}

helrm_status helrm_boot_matrix(const helrm_boot *bh, uint32_t which, helrm_ptmat **out)
{
    return guard(nullptr, [&] {
        HCHECK(out && which < 2, HELRM_E_INVAL, "which must be 0 or 1");
        *out = (helrm_ptmat *)BT(bh)->matrices()[which];
    });
}

helrm_status helrm_bootstrap(helrm_ctx *ctx, const helrm_evk *evk, const helrm_boot *b, const helrm_ct *in,
                             helrm_ct **out, helrm_ct **stages)
{
    if (out) *out = nullptr;
    if (stages)
        for (int i = 0; i < 5; i++) stages[i] = nullptr;
    return guard(ctx_or_null(ctx), [&] {
        HCHECK(out, HELRM_E_INVAL, "out is NULL");
        std::vector<Ciphertext *> st;
        std::unique_ptr<Ciphertext> y;
        try {
            y.reset(bootstrap(C(ctx), EVK(evk), BT(b), CT(in), stages ? &st : nullptr));
        } catch (...) {
            for (auto *p : st) delete p;
            throw;
        }
        for (size_t i = 0; i < st.size() && stages; i++) stages[i] = (helrm_ct *)st[i];
        *out = (helrm_ct *)y.release();
    });
}

void helrm_free(void *handle)
{
    if (!handle) return;
    Handle *h = (Handle *)handle;
    if (h->kind < KIND_CTX || h->kind > KIND_BOOT) return;
    delete h;
}

const char *helrm_last_error(const helrm_ctx *ctx)
{
    Ctx *c = ctx_or_null(ctx);
    return c ? c->last_error.c_str() : "invalid context";
}

const char *helrm_status_string(helrm_status s)
{
    switch (s) {
    case HELRM_OK: return "ok";
    case HELRM_E_INVAL: return "invalid argument";
    case HELRM_E_PARAM: return "unsupported parameters";
    case HELRM_E_LEVEL: return "level mismatch";
    case HELRM_E_SCALE: return "scale mismatch";
    case HELRM_E_NOKEY: return "missing key";
    case HELRM_E_NOMEM: return "out of device memory";
    case HELRM_E_CUDA: return "CUDA error";
    case HELRM_E_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

}  // extern "C"
