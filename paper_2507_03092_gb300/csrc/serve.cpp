// serve.cpp -- the served form: a request loop with continuous batching.
//
// Requests (shots of a compiled circuit with seeded streams) are queued by
// stab_serve_submit.  A scheduler thread admits queued requests in arrival
// order whenever a launch slot is free and the device memory the slots hold,
// plus what the request's slot still has to grow by, fits the HBM budget.
// Slots keep their buffers between requests (a smaller request reuses them
// without cudaFree / cudaMalloc); idle slots give theirs back only when
// nothing is in flight and the next request would not fit otherwise.
// Small-tableau requests that are waiting together are merged into one
// resident-engine launch (their shots become jobs of one persistent kernel);
// larger ones get a layered-engine launch.
// Each launch runs on its own CUDA stream, so requests admitted while others
// are on the GPU overlap with them on the device.  A host callback on the
// launch's stream stamps the completion time and frees the slot, and the
// scheduler admits the next requests.  Records are keyed by (seed, shot
// index), so a request's records are identical alone and in any mix.
#include "ctx.h"

#include <chrono>
#include <cstring>

namespace stab {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id;
    uint64_t circuit;
    uint32_t shots;
    uint64_t seed, shot_offset;
    uint64_t *d_record;
    uint64_t record_words;
    double t_submit, t_admit;
    size_t footprint;
    bool resident;
};

struct Slot {
    cudaStream_t stream = nullptr;
    bool busy = false;
    Batch work;
    MeasScratch ms;
    DevBuf ms_buf, jobs;
    unsigned int *counter = nullptr;
    std::vector<Request> reqs;     // requests of the launch in flight
    size_t held = 0;               // device bytes the slot's buffers hold
    int status = STAB_OK;
    struct ServeState *owner = nullptr;
};

static size_t slot_held(const Slot &s) { return s.work.cap + s.ms_buf.cap + s.jobs.cap; }

struct ServeState {
    stab_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::vector<std::unique_ptr<Slot>> slots;
    std::vector<stab_request_status> done;
    size_t held_bytes = 0;         // sum of the slots' held bytes
    uint64_t next_id = 1;
    size_t inflight = 0;
    bool stop = false;
    std::thread th;
    unsigned int *counters = nullptr;
};

static void CUDART_CB on_done(void *arg) {
    Slot *s = (Slot *)arg;
    ServeState *S = s->owner;
    const double t = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &r : s->reqs) {
        stab_request_status st{};
        st.req_id = r.id;
        st.status = s->status;
        st.shots = r.shots;
        st.t_submit = r.t_submit;
        st.t_admit = r.t_admit;
        st.t_done = t;
        S->done.push_back(st);
    }
    S->inflight -= s->reqs.size();
    s->reqs.clear();
    s->busy = false;
    S->cv.notify_all();
}

static size_t request_footprint(const HostProg &p, uint32_t shots, bool resident) {
    if (resident) return (size_t)shots * sizeof(ResJob);    // its job table (tableaux live in shared memory)
    const size_t mm = std::max<uint32_t>(1, layered_prog(p).dev.max_meas);
    return batch_bytes(p.n, shots) + (size_t)shots * mm * (4 * p.CW + 2);
}

static void scheduler(stab_ctx *ctx, ServeState *S) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->stop) break;
        Slot *slot = nullptr;
        for (auto &s : S->slots)
            if (!s->busy) { slot = s.get(); break; }
        if (!slot || S->queue.empty()) {
            S->cv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        // admit in arrival order: the head request, plus (for small tableaux)
        // the following queued resident requests that still fit
        std::vector<Request> take;
        size_t bytes = 0;
        const Request &head = S->queue.front();
        if (S->inflight >= S->cfg.max_inflight) {
            S->cv.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        auto extra_for = [&](size_t need) { return need > slot->held ? need - slot->held : (size_t)0; };
        if (S->held_bytes + extra_for(head.footprint) > S->cfg.hbm_budget_bytes) {
            bool any_busy = false;
            for (auto &s : S->slots) any_busy |= s->busy;
            if (any_busy) {
                S->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            // nothing in flight: idle slots give their buffers back, largest first
            // (cudaFree synchronises the device, which is idle)
            while (S->held_bytes + extra_for(head.footprint) > S->cfg.hbm_budget_bytes) {
                Slot *big = nullptr;
                for (auto &s : S->slots)
                    if (s.get() != slot && s->held && (!big || s->held > big->held)) big = s.get();
                if (!big) big = slot->held ? slot : nullptr;
                if (!big) break;
                batch_free(big->work);
                big->ms_buf.release();
                big->jobs.release();
                S->held_bytes -= big->held;
                big->held = 0;
            }
        }
        take.push_back(head);
        bytes += head.footprint;
        S->queue.pop_front();
        if (take[0].resident) {
            while (!S->queue.empty() && take.size() < S->cfg.max_batch_requests &&
                   S->inflight + take.size() < S->cfg.max_inflight) {
                const Request &nx = S->queue.front();
                if (!nx.resident || S->held_bytes + extra_for(bytes + nx.footprint) > S->cfg.hbm_budget_bytes) break;
                take.push_back(nx);
                bytes += nx.footprint;
                S->queue.pop_front();
            }
        }
        const double ta = now_s();
        for (auto &r : take) r.t_admit = ta;
        slot->busy = true;
        slot->reqs = take;
        slot->status = STAB_OK;
        S->inflight += take.size();
        lk.unlock();
        int rc = STAB_OK;
        {
            std::lock_guard<std::mutex> clk(ctx->mu);
            if (take[0].resident) {
                std::vector<stab_job_group> groups(take.size());
                for (size_t i = 0; i < take.size(); i++) {
                    stab_job_group &g = groups[i];
                    memset(&g, 0, sizeof(g));
                    g.circuit_id = take[i].circuit;
                    g.shots = take[i].shots;
                    g.streams.mode = STAB_STREAM_SEEDED;
                    g.streams.seed = take[i].seed;
                    g.streams.shot_offset = take[i].shot_offset;
                    g.d_record = take[i].d_record;
                    g.record_words = take[i].record_words;
                }
                rc = run_resident_groups(ctx, groups.data(), groups.size(), nullptr, slot->stream,
                                         slot->jobs, slot->counter);
            } else {
                const HostProg *p = find_prog(ctx, take[0].circuit);
                stab_streams st{};
                st.mode = STAB_STREAM_SEEDED;
                st.seed = take[0].seed;
                st.shot_offset = take[0].shot_offset;
                if (!p) rc = STAB_ERR_NOT_FOUND;
                else {
                    cudaMemsetAsync(take[0].d_record, 0, (size_t)take[0].shots * take[0].record_words * 8, slot->stream);
                    rc = run_layered_shots(ctx, *p, take[0].shots, st, take[0].d_record, take[0].record_words,
                                           slot->stream, slot->work, slot->ms, slot->ms_buf);
                }
            }
        }
        slot->status = rc;
        cudaError_t e = cudaLaunchHostFunc(slot->stream, on_done, slot);
        lk.lock();
        {
            const size_t h = slot_held(*slot);         // buffers may have grown for this launch
            S->held_bytes += h - slot->held;
            slot->held = h;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            lk.unlock();
            on_done(slot);
            lk.lock();
        }
    }
}

}  // namespace stab

using namespace stab;

extern "C" {

int stab_serve_start(stab_ctx *ctx, const stab_serve_config *cfg) {
    if (!ctx || !cfg) return fail(STAB_ERR_ARG, "context or config is NULL");
    if (ctx->serve) return fail(STAB_ERR_BUSY, "serving already started");
    if (!cfg->n_streams || !cfg->max_inflight || !cfg->hbm_budget_bytes)
        return fail(STAB_ERR_ARG, "n_streams, max_inflight and hbm_budget_bytes must be positive");
    cudaSetDevice(ctx->device);
    auto *S = new ServeState();
    S->cfg = *cfg;
    if (!S->cfg.max_batch_requests) S->cfg.max_batch_requests = 1;
    if (cudaMalloc(&S->counters, 256 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return fail(STAB_ERR_OOM, "cudaMalloc for serve counters failed");
    }
    const uint32_t ns = std::min<uint32_t>(cfg->n_streams, 256);
    for (uint32_t i = 0; i < ns; i++) {
        auto s = std::make_unique<Slot>();
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            const cudaError_t e = cudaGetLastError();
            for (auto &t : S->slots) cudaStreamDestroy(t->stream);   // nothing was launched on them
            cudaFree(S->counters);
            delete S;
            return cuda_fail(e, "cudaStreamCreate");
        }
        s->counter = S->counters + i;
        s->owner = S;
        S->slots.push_back(std::move(s));
    }
    ctx->serve = S;
    S->th = std::thread(scheduler, ctx, S);
    return STAB_OK;
}

int stab_serve_submit(stab_ctx *ctx, uint64_t circuit_id, uint32_t shots, uint64_t seed, uint64_t shot_offset,
                      uint64_t *d_record, uint64_t record_words, uint64_t *req_id) {
    if (!ctx || !ctx->serve) return fail(STAB_ERR_ARG, "serving not started");
    if (!req_id || !d_record || shots == 0) return fail(STAB_ERR_ARG, "bad request arguments");
    Request r{};
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        const HostProg *p = find_prog(ctx, circuit_id);
        if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id");
        if (record_words < p->info.record_words) return fail(STAB_ERR_STREAM_SHORT, "record buffer too short");
        // small tableaux go to the resident engine, where waiting requests
        // are merged into one launch (so a single request's shot count does
        // not decide); larger ones get their own layered launch sequence
        r.resident = prefer_resident(ctx, p->n, 1u << 20);
        if (!r.resident && !layered_supported(p->n, ctx->lc))
            return fail(STAB_ERR_UNSUPPORTED, "circuit too large for either engine");
        r.footprint = request_footprint(*p, shots, r.resident);
    }
    ServeState *S = ctx->serve;
    if (r.footprint > S->cfg.hbm_budget_bytes)
        return fail(STAB_ERR_OOM, "request footprint exceeds the serving HBM budget");
    r.circuit = circuit_id;
    r.shots = shots;
    r.seed = seed;
    r.shot_offset = shot_offset;
    r.d_record = d_record;
    r.record_words = record_words;
    r.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r.id = S->next_id++;
        S->queue.push_back(r);
        *req_id = r.id;
    }
    S->cv.notify_all();
    return STAB_OK;
}

int stab_serve_poll(stab_ctx *ctx, stab_request_status *done, size_t cap, size_t *n_done) {
    if (!ctx || !ctx->serve || !n_done || (cap && !done)) return fail(STAB_ERR_ARG, "bad poll arguments");
    ServeState *S = ctx->serve;
    std::lock_guard<std::mutex> lk(S->mu);
    const size_t k = std::min(cap, S->done.size());
    for (size_t i = 0; i < k; i++) done[i] = S->done[i];
    S->done.erase(S->done.begin(), S->done.begin() + (long)k);
    *n_done = k;
    return STAB_OK;
}

int stab_serve_drain(stab_ctx *ctx, double timeout_s) {
    if (!ctx || !ctx->serve) return fail(STAB_ERR_ARG, "serving not started");
    ServeState *S = ctx->serve;
    const double t_end = now_s() + timeout_s;
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->queue.empty() || S->inflight > 0) {
        if (now_s() > t_end) return fail(STAB_ERR_TIMEOUT, "requests still pending after the drain timeout");
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
    return STAB_OK;
}

int stab_serve_stop(stab_ctx *ctx) {
    if (!ctx || !ctx->serve) return fail(STAB_ERR_ARG, "serving not started");
    ServeState *S = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(ctx->device);
    for (auto &s : S->slots) {
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
        batch_free(s->work);
        s->ms_buf.release();
        s->jobs.release();
    }
    cudaFree(S->counters);
    ctx->serve = nullptr;
    delete S;
    return STAB_OK;
}

}  // extern "C"
