// model.cuh -- the compiled DLRM (layers, packed embedding, masks) shared by
// the one-query path (dlrm.cu) and the batched path (batch.cu).
#pragma once

#include <algorithm>
#include <array>

#include "core.cuh"

namespace helrm {

constexpr int DIM = 16;

// A polynomial evaluation fixed for an input level and scale (poly.cu): the
// products that form the needed powers, the simulated scale of each power,
// the integer constant of each term as per-prime Montgomery residues, and the
// constant term as plain residues.
struct ActPlan {
    std::vector<double> a;                      // a_0 .. a_d
    std::vector<std::array<int, 3>> tree;       // (k, a, b): x^k = x^a x^b, increasing k
    std::map<int, double> pw_scale;             // scale of x^k
    int in_level = 0, level_c = 0, out_level = 0;
    double in_scale = 0, out_scale = 0;
    struct Term {
        int k;
        double scale;                           // scale of a_k x^k before the rescale
        DevMem mont;                            // [c_k]_q R mod q per prime id
    };
    std::vector<Term> terms;
    DevMem a0;                                  // [round(a_0 out_scale)]_q per prime id (empty: a_0 = 0)
};
int poly_depth(int d);
// per-prime residues of an integer (Montgomery form when mont), as a device table indexed by prime id
DevMem int_table(Ctx *c, i64 v, bool mont);
// the same for an integer-valued double of any finite size (the exact integer it holds)
DevMem int_table_f(Ctx *c, double v, bool mont);
double round_half_away(double v);
ActPlan *act_plan(Ctx *c, const std::vector<double> &a, int level, double scale, double target);
// the plan's polynomial on every query's ciphertext (batch.cu); evk[q]: the
// relinearisation key of query q
std::vector<Ciphertext *> poly_b(Ctx *c, const std::vector<const EvalKey *> &evk,
                                 const std::vector<const Ciphertext *> &x, const ActPlan &plan);
Ciphertext *ct_poly_eval(Ctx *c, const EvalKey *evk, const Ciphertext *x, const std::vector<double> &a,
                         double target);

// Bootstrapping of a ciphertext whose real slots are periodic with period n_s
// (boot.cu): ModRaise, SubSum, CoeffToSlot (one product and the conjugate
// of its output), EvalMod (cosine fit, r double angles), SlotToCoeff.
struct Boot : Handle {
    Ctx *ctx;
    int n_s = 0, K = 0, r = 0, degree = 0, log2_boost = 0, cts_levels = 1;
    int level_top = 0, level_stc = 0, level_out = 0;
    double s_ref = 0, eval_scale = 0;
    std::vector<double> coeffs;                 // the cosine polynomial, power basis in y
    std::unique_ptr<PtMatrix> cts_a;            // CoeffToSlot, at level_top
    std::unique_ptr<PtMatrix> stc;              // SlotToCoeff at level_stc
    std::vector<int> subsum_steps;
    DevMem boost_mont;                          // 2^b per prime id, Montgomery form
    // fixed at creation (no host synchronisation while bootstrapping, so a
    // bootstrap can be captured in a CUDA graph): the CoeffToSlot output scale,
    // the EvalMod constants and polynomial plan, the SlotToCoeff scale factor
    double s_cts = 0, s_eval = 0, c_out = 0;
    DevMem c_shift;                             // round(-s_cts / (4 2^r)), plain residues per prime id
    std::unique_ptr<ActPlan> plan;              // the cosine polynomial at (L - cts_levels, s_cts)
    std::vector<DevMem> c_double;               // round(-scale) after each double angle's product
    Boot(Ctx *c) : Handle(KIND_BOOT), ctx(c) {}
    // the declared scale of the output for an input of scale in_scale
    double out_scale(double in_scale) const { return c_out * (in_scale / s_ref); }
    std::vector<int> rotations() const;
    std::vector<PtMatrix *> matrices() const { return {cts_a.get(), stc.get()}; }
};
struct BootDesc {
    int n_s, K, r, degree, log2_boost, cts_levels;
    double s_ref, eval_scale;
    std::vector<double> coeffs;   // empty: the library's Chebyshev fit
};
Boot *boot_create(Ctx *c, const BootDesc &d);
std::vector<double> boot_cos_fit(int K, int r, int degree);
// stages (optional, 5 entries): raised, subsum, CoeffToSlot, EvalMod, output
// (the caller owns them; the output is also returned)
Ciphertext *bootstrap(Ctx *c, const EvalKey *evk, const Boot *b, const Ciphertext *in,
                      std::vector<Ciphertext *> *stages = nullptr);

struct SelSeg {
    int t, j, off, width;
};

struct Emb : Handle {
    Ctx *ctx;
    std::vector<u64> cards;
    int base = 0, dim = 0, width = 0, in_pad = 0, out_pad = 0;
    u64 threshold = 0;   // tables with more rows are digit-decomposed
    std::vector<SelSeg> layout;
    std::unique_ptr<PtMatrix> pm;                    // the lookup matrix (selector within one ciphertext)
    // a selector wider than the slot count spans ceil(width / n) ciphertexts:
    // chunk c holds columns [c n, min((c + 1) n, width)) and has its own matrix
    std::vector<std::unique_ptr<PtMatrix>> chunks;   // (pm is then null)
    DevMem d_tab;   // int [T][3]: card (clamped), offset, digits
    Emb(Ctx *c) : Handle(KIND_EMB), ctx(c) {}
};

struct Layer {
    std::unique_ptr<PtMatrix> pm;
    std::unique_ptr<Plaintext> bias;
    bool square = false;                    // an activation follows: x^2, or act (a polynomial)
    std::unique_ptr<ActPlan> act;           // the activation polynomial without a_0 (null: x^2)
    std::unique_ptr<Plaintext> act_const;   // a_0 on the layer's real outputs (null: none)
};

struct Model : Handle {
    Ctx *ctx;
    int n_dense = 0, interaction = 0, T = 0, B = 0, Bp = 0, S = 0;
    int lvl_dense = 0, lvl_sel = 0, lvl_z = 0, lvl_u = 0, p_dense = 0, W_z = 0, W2 = 0, W_u = 0;
    double mask_scale = 0;
    std::vector<Layer> bottom, top;
    std::unique_ptr<Emb> emb;
    std::unique_ptr<Plaintext> ones;
    std::vector<std::unique_ptr<Plaintext>> masks;
    std::vector<double> act;   // the activation polynomial a_0 .. a_d (empty: x^2)
    // bootstraps: before bottom layer i (boot_b[i], i >= 1), on z before the
    // interaction (boot_z), before top layer i (boot_t[i], i >= 1); each lifts
    // its input (level 0, the end of a segment) and drops it to lvl_next
    struct BootPoint {
        std::unique_ptr<Boot> b;
        int lvl_next = 0;
    };
    std::vector<BootPoint> boot_b, boot_t;
    BootPoint boot_z;
    int lvl_h = 0;   // level of z = h + e (lvl_z unless z is bootstrapped)
    Model(Ctx *c) : Handle(KIND_MODEL), ctx(c) {}
    // the bootstrap points in the order the inference meets them
    std::vector<const BootPoint *> boot_points() const
    {
        std::vector<const BootPoint *> v;
        for (auto &x : boot_b)
            if (x.b) v.push_back(&x);
        if (boot_z.b) v.push_back(&boot_z);
        for (auto &x : boot_t)
            if (x.b) v.push_back(&x);
        return v;
    }
    bool has_boot() const { return !boot_points().empty(); }

    // the lookup's matrices: one, or one per ciphertext of a wide selector
    std::vector<PtMatrix *> emb_mats() const
    {
        std::vector<PtMatrix *> v;
        if (emb->pm) v.push_back(emb->pm.get());
        for (auto &ch : emb->chunks) v.push_back(ch.get());
        return v;
    }
    int n_sel() const { return (int)emb_mats().size(); }
    std::vector<std::unique_ptr<Plaintext> *> plaintexts()
    {
        std::vector<std::unique_ptr<Plaintext> *> out;
        auto layer = [&](Layer &l) {
            for (auto &p : l.pm->pts) out.push_back(&p);
            out.push_back(&l.bias);
            if (l.act_const) out.push_back(&l.act_const);
        };
        for (auto &l : bottom) layer(l);
        for (PtMatrix *pm : emb_mats())
            for (auto &p : pm->pts) out.push_back(&p);
        if (interaction == 0) {
            out.push_back(&ones);
            for (auto &m : masks) out.push_back(&m);
        }
        for (auto &l : top) layer(l);
        for (const BootPoint *bp : boot_points())
            for (PtMatrix *pm : bp->b->matrices())
                for (auto &p : pm->pts) out.push_back(&p);
        return out;
    }
    std::vector<int> rotations() const
    {
        std::vector<int> st;
        auto addv = [&](const std::vector<int> &v) { st.insert(st.end(), v.begin(), v.end()); };
        for (auto &l : bottom) addv(l.pm->rotations());
        for (PtMatrix *pm : emb_mats()) addv(pm->rotations());
        if (interaction == 0) {
            st.push_back(-DIM * Bp);
            for (int s = 1; s <= S; s++) st.push_back(DIM * s);
        }
        for (auto &l : top) addv(l.pm->rotations());
        for (const BootPoint *bp : boot_points()) addv(bp->b->rotations());
        std::sort(st.begin(), st.end());
        st.erase(std::unique(st.begin(), st.end()), st.end());
        return st;
    }
};

// ct_sel: the model's n_sel() selector ciphertexts
Ciphertext *model_infer(Ctx *c, const EvalKey *evk, const Model *m, const Ciphertext *ct_dense,
                        const std::vector<const Ciphertext *> &ct_sel);


}  // namespace helrm
