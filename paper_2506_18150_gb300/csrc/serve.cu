// serve.cu -- the request loop: continuous batching over lockstep batches.
//
// Clients register once (model + evaluation keys, which stay resident in
// HBM).  helrm_server_run replays a trace of timed requests (ciphertexts
// already on the device) through a loop that
//  * moves every request whose arrival time has passed into a pending queue;
//  * whenever one of the server's batch slots (one CUDA stream each) is free
//    and the memory budget admits it, takes the oldest pending request and up
//    to max_batch - 1 more pending requests of the same model, and launches
//    them as one lockstep batch (batch.cu) on that slot's stream; batches on
//    different slots overlap on the device, so requests that arrive while
//    others are on the GPU start as soon as a slot and memory free up;
//  * polls each slot's completion event, and on completion records the
//    latency (completion - arrival) of every request of the batch and hands
//    back its encrypted logit.
// A batch of one request runs the one-query path (helrm_infer), so a server
// with one slot and max_batch = 1 is the plain one-request-at-a-time path.
// A model whose selector is wider than the slots brings n_sel selector
// ciphertexts per request; its batches carry them query by query.
//
// Time is the host's steady clock.  When nothing is pending or in flight the
// loop skips ahead to the next arrival instead of sleeping (the idle GPU has
// nothing to do meanwhile), so sparse traces replay quickly; latencies are
// unaffected.  Admission control: each model's per-query device footprint is
// measured on its first request, which runs alone; a batch is shrunk until the bytes in flight plus its footprint fit
// the budget (the one given at creation, and the room left under the
// context's memory cap when one is set); a single request is always admitted
// when nothing else is in flight.
#include <algorithm>
#include <chrono>
#include <deque>
#include <thread>

#include "model.cuh"

namespace helrm {

struct Batch;
Batch *batch_create(Ctx *c, const Model *m, const std::vector<const EvalKey *> &evk);
std::vector<Ciphertext *> model_infer_batch(Ctx *c, const Batch *bt, const std::vector<const Ciphertext *> &ct_dense,
                                            const std::vector<const Ciphertext *> &ct_sel);
void batch_destroy(Batch *b);

struct Server : Handle {
    Ctx *ctx;
    int n_slots = 1, max_batch = 1;
    u64 budget = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    struct Client {
        const Model *m;
        const EvalKey *evk;
    };
    std::vector<Client> clients;
    std::map<const Model *, u64> per_query;   // observed device bytes per query of each model
    Server(Ctx *c) : Handle(KIND_SERVER), ctx(c) {}
    ~Server() override
    {
        for (auto s : streams) cudaStreamSynchronize(s);
        for (auto e : events) cudaEventDestroy(e);
        for (auto s : streams) cudaStreamDestroy(s);
    }
};

Server *server_create(Ctx *c, int n_slots, int max_batch, u64 budget)
{
    HCHECK(n_slots >= 1 && n_slots <= 16 && max_batch >= 1 && max_batch <= 256, HELRM_E_INVAL,
           "server needs 1..16 slots and a batch size of 1..256");
    std::unique_ptr<Server> s(new Server(c));
    s->n_slots = n_slots;
    s->max_batch = max_batch;
    s->budget = budget;
    for (int i = 0; i < n_slots; i++) {
        cudaStream_t st;
        cudaEvent_t ev;
        CUDA_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CUDA_CHECK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        s->streams.push_back(st);
        s->events.push_back(ev);
    }
    return s.release();
}

u32 server_add_client(Server *s, const Model *m, const EvalKey *evk)
{
    s->clients.push_back({m, evk});
    return (u32)s->clients.size() - 1;
}

// Selector ciphertexts of a trace: request r brings the n_sel of its
// client's model (one unless the selector is wider than the slots), request
// after request.  Checks the client ids; returns the total.
u32 server_sel_count(const Server *s, u32 n, const u32 *client)
{
    u64 total = 0;
    for (u32 r = 0; r < n; r++) {
        HCHECK(client[r] < s->clients.size(), HELRM_E_INVAL, "request names an unknown client");
        total += (u64)s->clients[client[r]].m->n_sel();
    }
    HCHECK(total < (1ull << 31), HELRM_E_INVAL, "too many selector ciphertexts");
    return (u32)total;
}

namespace {

struct InFlight {
    int slot = -1;
    std::vector<u32> reqs;
    Batch *batch = nullptr;
    std::vector<Ciphertext *> out;
    const Model *model = nullptr;
    u64 bytes = 0;        // admitted footprint
    bool measure = false; // first batch of its model: its footprint is observed
    u64 base = 0;         // bytes held when it was launched
};

using Clock = std::chrono::steady_clock;

}  // namespace

void server_run(Server *s, u32 n, const double *arrival, const u32 *client, const Ciphertext *const *ct_dense,
                const Ciphertext *const *ct_sel, Ciphertext **out, double *latency_ms, helrm_serve_stats *st)
{
    Ctx *c = s->ctx;
    server_sel_count(s, n, client);
    std::vector<u32> sel_off(n + 1, 0);   // request r's selectors: ct_sel[sel_off[r] .. sel_off[r + 1])
    for (u32 r = 0; r < n; r++) {
        HCHECK(r == 0 || arrival[r] >= arrival[r - 1], HELRM_E_INVAL, "arrivals must be sorted");
        sel_off[r + 1] = sel_off[r] + (u32)s->clients[client[r]].m->n_sel();
    }
    auto sels = [&](u32 r) {
        return std::vector<const Ciphertext *>(ct_sel + sel_off[r], ct_sel + sel_off[r + 1]);
    };
    CUDA_CHECK(cudaStreamSynchronize(c->stream));   // the requests' ciphertexts are ready
    const cudaStream_t home = c->stream;
    std::deque<u32> pending;
    std::vector<InFlight> fl(s->n_slots);
    std::vector<char> busy(s->n_slots, 0);
    u32 next = 0, done = 0, batches = 0, max_seen = 0, max_inflight = 0;
    double sum_batch = 0, skipped = 0;
    u64 inflight_bytes = 0;
    const auto t0 = Clock::now();
    auto vnow = [&] { return std::chrono::duration<double>(Clock::now() - t0).count() + skipped; };
    auto finish = [&](int k, double t) {
        InFlight &f = fl[k];
        c->stream = s->streams[k];
        if (f.measure) {   // first batch of this model (it ran alone): learn its per-query footprint
            const u64 used = c->mem_peak > f.base ? c->mem_peak - f.base : 0;
            s->per_query[f.model] = std::max<u64>(used / f.reqs.size(), 1);
        }
        for (size_t i = 0; i < f.reqs.size(); i++) {
            const u32 r = f.reqs[i];
            latency_ms[r] = 1000.0 * (t - arrival[r]);
            out[r] = f.out[i];
        }
        if (f.batch) batch_destroy(f.batch);
        c->stream = home;
        done += (u32)f.reqs.size();
        inflight_bytes -= std::min(inflight_bytes, f.bytes);
        f = InFlight();
        busy[k] = 0;
    };
    try {
        while (done < n) {
            double t = vnow();
            while (next < n && arrival[next] <= t) pending.push_back(next++);
            for (int k = 0; k < s->n_slots; k++)
                if (busy[k]) {
                    cudaError_t q = cudaEventQuery(s->events[k]);
                    if (q == cudaSuccess)
                        finish(k, t);
                    else if (q != cudaErrorNotReady)
                        CUDA_CHECK(q);
                }
            int n_busy = 0;
            for (int k = 0; k < s->n_slots; k++) n_busy += busy[k];
            while (!pending.empty() && n_busy < s->n_slots) {
                const Model *m = s->clients[client[pending.front()]].m;
                const bool known = s->per_query.count(m) != 0;
                if (!known && n_busy) break;   // ... to measure its footprint
                std::vector<u32> take;
                const int cap = known ? s->max_batch : 1;   // a model's first batch is one request, run alone
                for (auto it = pending.begin(); it != pending.end() && (int)take.size() < cap; ++it)
                    if (s->clients[client[*it]].m == m) take.push_back(*it);
                u64 need = known ? s->per_query[m] * take.size() : 0;
                u64 budget = s->budget;   // bytes that in-flight batches may hold
                if (c->mem_cap) {
                    const u64 room = c->mem_cap > c->mem_in_use ? c->mem_cap - c->mem_in_use : 0;
                    budget = budget ? std::min(budget, room) : std::max<u64>(room, 1);
                }
                if (budget && known) {
                    const u64 per = s->per_query[m];
                    while (!take.empty() && inflight_bytes + per * take.size() > budget) take.pop_back();
                    if (take.empty() && n_busy == 0) take.push_back(pending.front());   // always make progress
                    need = per * take.size();
                }
                if (take.empty()) break;
                int k = 0;
                while (busy[k]) k++;
                InFlight &f = fl[k];
                f.slot = k;
                f.reqs = take;
                f.model = m;
                f.bytes = need;
                f.measure = !known;
                f.base = c->mem_in_use;
                if (!known) c->mem_peak = c->mem_in_use;
                c->stream = s->streams[k];
                busy[k] = 1;   // from here on the slot owns whatever was launched
                if (take.size() == 1) {
                    const Server::Client &cl = s->clients[client[take[0]]];
                    f.out.push_back(model_infer(c, cl.evk, m, ct_dense[take[0]], sels(take[0])));
                } else {
                    std::vector<const EvalKey *> ev;
                    std::vector<const Ciphertext *> d, sl;
                    for (u32 r : take) {
                        ev.push_back(s->clients[client[r]].evk);
                        d.push_back(ct_dense[r]);
                        for (const Ciphertext *x : sels(r)) sl.push_back(x);
                    }
                    f.batch = batch_create(c, m, ev);
                    f.out = model_infer_batch(c, f.batch, d, sl);
                }
                CUDA_CHECK(cudaEventRecord(s->events[k], s->streams[k]));
                c->stream = home;
                n_busy++;
                inflight_bytes += need;
                batches++;
                sum_batch += (double)take.size();
                max_seen = std::max<u32>(max_seen, (u32)take.size());
                max_inflight = std::max<u32>(max_inflight, (u32)n_busy);
                for (u32 r : take) pending.erase(std::find(pending.begin(), pending.end(), r));
            }
            if (n_busy == 0 && pending.empty() && next < n) {
                skipped += arrival[next] - vnow();   // idle: jump to the next arrival
                continue;
            }
            if (n_busy) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    } catch (...) {
        // release everything: the batches still in flight and the logits handed out so far
        for (int k = 0; k < s->n_slots; k++)
            if (busy[k]) {
                cudaStreamSynchronize(s->streams[k]);
                c->stream = s->streams[k];
                for (auto *p : fl[k].out) delete p;
                if (fl[k].batch) batch_destroy(fl[k].batch);
            }
        c->stream = home;
        for (u32 r = 0; r < n; r++) {
            delete out[r];
            out[r] = nullptr;
        }
        throw;
    }
    const double makespan = vnow();
    if (st) {
        std::vector<double> lat(latency_ms, latency_ms + n);
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) { return lat.empty() ? 0.0 : lat[std::min<size_t>(lat.size() - 1, (size_t)(p * (lat.size() - 1) + 0.5))]; };
        double sum = 0;
        for (double x : lat) sum += x;
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->mean_ms = n ? sum / n : 0;
        st->max_ms = lat.empty() ? 0 : lat.back();
        st->makespan_s = makespan;
        st->throughput = makespan > 0 ? n / makespan : 0;
        st->n_batches = batches;
        st->mean_batch = batches ? sum_batch / batches : 0;
        st->max_batch = max_seen;
        st->max_inflight = max_inflight;
    }
}

}  // namespace helrm
