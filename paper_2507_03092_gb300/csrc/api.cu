// api.cu -- implementation of the C ABI declared in include/stab.h.
#include "ctx.h"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace stab {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return STAB_ERR_CUDA;
}

void smem_attr_once(int slot, const void *func, int bytes) {
    static std::mutex mu;
    static uint64_t done[32];            // bit d of done[slot]: set on device d
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || slot < 0 || slot >= 32) {
        cudaGetLastError();
        cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        return;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (done[slot] >> dev & 1u) return;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
        done[slot] |= 1ull << dev;
    else
        cudaGetLastError();
}

int DevBuf::ensure(size_t bytes) {
    if (bytes <= cap) return STAB_OK;
    release();
    size_t want = std::max(bytes, cap * 3 / 2);
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        cap = 0;
        return fail(STAB_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    cap = want;
    return STAB_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

cudaEvent_t KernelProf::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void KernelProf::begin(uint32_t kind, cudaStream_t s, Rec &r) {
    r.kind = kind;
    r.e0 = take();
    r.e1 = take();
    r.bytes = 0.0;
    cudaEventRecord(r.e0, s);
}

void KernelProf::end(Rec &r, cudaStream_t s, double b) {
    cudaEventRecord(r.e1, s);
    r.bytes = b;
    pending.push_back(r);
}

int KernelProf::collect() {
    for (auto &r : pending) {
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e) return cuda_fail(e, "waiting for a profiling event");
        float t = 0.f;
        cudaEventElapsedTime(&t, r.e0, r.e1);
        n[r.kind]++;
        ms[r.kind] += t;
        bytes[r.kind] += r.bytes;
        pool.push_back(r.e0);
        pool.push_back(r.e1);
    }
    pending.clear();
    return STAB_OK;
}

const HostProg *find_prog(stab_ctx *ctx, uint64_t id) {
    auto it = ctx->progs.find(id);
    return it == ctx->progs.end() ? nullptr : it->second.get();
}

DevStreams to_dev(const stab_streams &s) {
    DevStreams d{};
    d.mode = s.mode;
    d.seed = s.seed;
    d.shot_offset = s.shot_offset;
    d.coins = (const unsigned long long *)s.coins;
    d.coin_stride = s.coin_words;
    d.noise = s.noise;
    d.noise_stride = s.noise_words;
    return d;
}

int check_streams(const HostProg &p, const stab_streams *s, uint32_t shots) {
    if (!s) return fail(STAB_ERR_ARG, "streams is NULL");
    if (s->mode == STAB_STREAM_SEEDED) return STAB_OK;
    if (s->mode != STAB_STREAM_BUFFER) return fail(STAB_ERR_ARG, "unknown stream mode");
    if (shots == 0) return STAB_OK;
    if (p.info.n_coin > 0) {
        if (!s->coins) return fail(STAB_ERR_ARG, "coin buffer is NULL");
        if (s->coin_words < p.info.coin_words)
            return fail(STAB_ERR_STREAM_SHORT, "coin stream has " + std::to_string(s->coin_words) +
                                                   " words per shot, circuit needs " +
                                                   std::to_string(p.info.coin_words));
    }
    if (p.info.n_noise_words > 0) {
        if (!s->noise) return fail(STAB_ERR_ARG, "noise buffer is NULL");
        if (s->noise_words < p.info.n_noise_words)
            return fail(STAB_ERR_STREAM_SHORT, "noise stream has " + std::to_string(s->noise_words) +
                                                   " words per shot, circuit needs " +
                                                   std::to_string(p.info.n_noise_words));
    }
    return STAB_OK;
}

static int ensure_ms(MeasScratch &ms, DevBuf &buf, const HostProg &p, uint32_t count) {
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t mm = std::max<uint32_t>(1, p.dev.max_meas);
    const size_t words = mm * p.CW * count, items = mm * count;
    const size_t mxs_b = 2 * (size_t)XSCAP * items, mxn_b = items, mxver_b = 4 * items;
    const size_t rowver_b = 4 * (size_t)32 * p.H * count;
    const size_t qmap_b = 2 * (size_t)p.n * count;
    const size_t piv_b = 4 * items, bsz_b = 4 * items, stale_b = items;
    const size_t sup_b = 2 * (size_t)SUPCAP * items;
    const size_t pwl_b = 2 * (size_t)WaveCaps::WCAP_MAX * PWCAP * count;
    const size_t flips_b = 4 * 2 * items;
    const size_t ev_b = 4 * (size_t)std::max<uint32_t>(1, p.dev.ev_total) * count;
    const size_t cnt_b = 4 * (size_t)std::max<size_t>(1, p.layers.size()) * count;
    const size_t bytes = up(4 * words) + up(2 * items) + up(mxs_b) + up(mxn_b) + up(mxver_b) + up(rowver_b) +
                         up(ev_b) + up(cnt_b) +
                         up(qmap_b) + up(piv_b) + up(bsz_b) + up(stale_b) + up(sup_b) + up(pwl_b) +
                         up(flips_b) + up(cnt_b) + up(sizeof(CallArgs));
    int rc = buf.ensure(bytes);
    if (rc) return rc;
    char *b = (char *)buf.p;
    ms.cols = (uint32_t *)b; b += up(4 * words);
    ms.stat = (uint8_t *)b;
    ms.out = ms.stat + items; b += up(2 * items);
    ms.mxs = (uint16_t *)b; b += up(mxs_b);
    ms.mxn = (uint8_t *)b; b += up(mxn_b);
    ms.mxver = (uint32_t *)b; b += up(mxver_b);
    ms.rowver = (uint32_t *)b; b += up(rowver_b);
    ms.ev = (uint32_t *)b; b += up(ev_b);
    ms.ev_cnt = (uint32_t *)b; b += up(cnt_b);
    ms.qmap = (uint16_t *)b; b += up(qmap_b);
    ms.mpiv = (uint32_t *)b; b += up(piv_b);
    ms.mbsz = (uint32_t *)b; b += up(bsz_b);
    ms.mstale = (uint8_t *)b; b += up(stale_b);
    ms.msup = (uint16_t *)b; b += up(sup_b);
    ms.pwl = (uint16_t *)b; b += up(pwl_b);
    ms.flips = (uint32_t *)b; b += up(flips_b);
    ms.flip_cnt = (uint32_t *)b; b += up(cnt_b);
    ms.call = (CallArgs *)b;
    ms.cap_words = words;
    ms.cap_items = items;
    return STAB_OK;
}

stab_tune default_tune(const stab_ctx *ctx, uint32_t n) {
    stab_tune t{};
    const uint32_t CW = 2 * ((n + 31) / 32);
    (void)CW;
    t.words_per_thread = CW >= 8 ? 2 : 1;
    t.group_threads = n <= 64 ? 32 : (n <= 256 ? 64 : 128);
    const size_t per = resident_smem_per_tableau(n);
    uint32_t tpc = std::max<uint32_t>(1, 256 / t.group_threads);
    while (tpc > 1 && per * tpc > ctx->lc.smem_optin) tpc--;
    if (t.group_threads > 32) tpc = std::min<uint32_t>(tpc, 15);
    t.tableaux_per_cta = tpc;
    while (t.tableaux_per_cta > 1 && !resident_shape_ok(n, t, ctx->lc)) t.tableaux_per_cta--;
    return t;
}

stab_tune lookup_tune(const stab_ctx *ctx, uint32_t n) {
    auto it = ctx->tune.find((n + 31) / 32);
    if (it != ctx->tune.end()) return it->second;
    return default_tune(ctx, n);
}

// One device allocation holds every array of a compiled program, followed by
// its DevProg descriptor (used by the resident engine's job table).
static constexpr int PROG_ARRAYS = 9;
static size_t prog_layout(const HostProg &P, size_t off[PROG_ARRAYS + 1]) {
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t sz[PROG_ARRAYS] = {P.layers.size() * sizeof(Layer), P.gitems.size() * sizeof(GItem),
                                    P.mitems.size() * sizeof(MItem), P.thr.size() * sizeof(Thr),
                                    P.sitems.size() * sizeof(SItem), P.item_layer.size() * sizeof(uint32_t),
                                    P.mfactors.size() * sizeof(uint32_t), P.sab.size() * sizeof(uint32_t),
                                    P.layers.size()};
    size_t o = 0;
    for (int k = 0; k < PROG_ARRAYS; k++) {
        off[k] = o;
        o += up(sz[k] + 1);
    }
    off[PROG_ARRAYS] = o;
    return o + up(sizeof(DevProg));
}

static void free_prog(HostProg &P) {
    if (P.lay) free_prog(*P.lay);
    prog_graphs_free(P);
    if (P.rand_ev) {
        cudaEventSynchronize(P.rand_ev);
        cudaEventDestroy(P.rand_ev);
    }
    if (P.rand_host) cudaFreeHost(P.rand_host);
    P.rand_ev = nullptr;
    P.rand_host = nullptr;
    if (P.dmem) cudaFree(P.dmem);
    P.dmem = nullptr;
}

static int upload_prog(HostProg &P) {
    size_t off[PROG_ARRAYS + 1];
    const size_t total = prog_layout(P, off);
    if (cudaMalloc(&P.dmem, total) != cudaSuccess) {
        cudaGetLastError();
        P.dmem = nullptr;
        return fail(STAB_ERR_OOM, "cudaMalloc for the compiled circuit failed");
    }
    char *b = (char *)P.dmem;
    P.dev.layers = (const Layer *)(b + off[0]);
    P.dev.gitems = (const GItem *)(b + off[1]);
    P.dev.mitems = (const MItem *)(b + off[2]);
    P.dev.thr = (const Thr *)(b + off[3]);
    P.dev.sitems = (const SItem *)(b + off[4]);
    P.dev.item_layer = (const uint32_t *)(b + off[5]);
    P.dev.mfactors = (const uint32_t *)(b + off[6]);
    P.dev.sab = (const uint32_t *)(b + off[7]);
    P.dev.layer_rand = (uint8_t *)(b + off[8]);
    const void *src[PROG_ARRAYS - 1] = {P.layers.data(), P.gitems.data(), P.mitems.data(), P.thr.data(),
                                        P.sitems.data(), P.item_layer.data(), P.mfactors.data(), P.sab.data()};
    const size_t sz[PROG_ARRAYS - 1] = {P.layers.size() * sizeof(Layer), P.gitems.size() * sizeof(GItem),
                                        P.mitems.size() * sizeof(MItem), P.thr.size() * sizeof(Thr),
                                        P.sitems.size() * sizeof(SItem), P.item_layer.size() * sizeof(uint32_t),
                                        P.mfactors.size() * sizeof(uint32_t), P.sab.size() * sizeof(uint32_t)};
    cudaError_t e = cudaMemset(b + off[8], 0, P.layers.size() + 1);   // no layer marked yet
    for (int k = 0; k < PROG_ARRAYS - 1 && !e; k++)
        if (sz[k]) e = cudaMemcpy(b + off[k], src[k], sz[k], cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b + off[PROG_ARRAYS], &P.dev, sizeof(DevProg), cudaMemcpyHostToDevice);
    if (e) return cuda_fail(e, "uploading the compiled circuit");
    if (P.lay) return upload_prog(*P.lay);
    return STAB_OK;
}

const DevProg *prog_desc(const HostProg &P) {
    size_t off[PROG_ARRAYS + 1];
    prog_layout(P, off);
    return (const DevProg *)((char *)P.dmem + off[PROG_ARRAYS]);
}

int run_layered_shots(stab_ctx *ctx, const HostProg &user_prog, uint32_t shots, const stab_streams &st,
                      uint64_t *d_record, uint64_t record_words, cudaStream_t s, Batch &work,
                      MeasScratch &ms, DevBuf &ms_buf) {
    const HostProg &p = layered_prog(user_prog);
    if (!layered_supported(p.n, ctx->lc))
        return fail(STAB_ERR_UNSUPPORTED, "n = " + std::to_string(p.n) + " exceeds the layered engine's shared-memory slice");
    // chunk so the batch stays within a fixed device budget
    const size_t per = batch_bytes(p.n, 1);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    size_t budget = std::min<size_t>((size_t)16 << 30, free_b / 3 + work.cap);
    // grid.y indexes the tableau: at most 65535 per launch
    uint32_t chunk = (uint32_t)std::max<size_t>(1, std::min<size_t>({(size_t)shots, budget / per, (size_t)65535}));
    if (work.n != p.n || work.count < chunk) {
        std::string err;
        int rc = batch_alloc(work, p.n, chunk, &err);
        if (rc) return fail(rc, err);
    }
    for (uint32_t s0 = 0; s0 < shots; s0 += chunk) {
        const uint32_t cnt = std::min(chunk, shots - s0);
        Batch b = work;
        b.count = cnt;
        int rc = ensure_ms(ms, ms_buf, p, cnt);
        if (rc) return rc;
        cudaError_t e = layered_init(b, s, &ctx->prof);
        if (e) return cuda_fail(e, "layered init");
        DevStreams ds = to_dev(st);
        if (st.mode == STAB_STREAM_SEEDED) ds.shot_offset += s0;
        else {
            if (ds.coins) ds.coins += (size_t)s0 * ds.coin_stride;
            if (ds.noise) ds.noise += (size_t)s0 * ds.noise_stride;
        }
        GraphSlot *gsl = (s == ctx->stream && graph_slot_init(ctx->gslot) == 0) ? &ctx->gslot : nullptr;
        e = layered_run(p, b, ms, ds, (unsigned long long *)(d_record + (size_t)s0 * record_words),
                        record_words, ctx->d_err, ctx->lc, s, &ctx->prof, ctx->d_stats, gsl, true);
        if (e) return cuda_fail(e, "layered run");
        work.rm_valid = b.rm_valid;
    }
    return STAB_OK;
}

int run_resident_groups(stab_ctx *ctx, const stab_job_group *groups, size_t n_groups,
                        const stab_tune *force, cudaStream_t s, DevBuf &jobs, unsigned int *counter) {
    uint64_t total = 0;
    uint32_t max_n = 0;
    std::vector<std::pair<uint64_t, ResJob>> hj;
    for (size_t gi = 0; gi < n_groups; gi++) {
        const stab_job_group &G = groups[gi];
        const HostProg *p = find_prog(ctx, G.circuit_id);
        if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id " + std::to_string(G.circuit_id));
        if (!resident_supported(p->n, ctx->lc))
            return fail(STAB_ERR_UNSUPPORTED, "n = " + std::to_string(p->n) + " does not fit the resident engine");
        int rc = check_streams(*p, &G.streams, G.shots);
        if (rc) return rc;
        if (G.shots && !G.d_record) return fail(STAB_ERR_ARG, "record buffer is NULL");
        if (G.record_words < p->info.record_words)
            return fail(STAB_ERR_STREAM_SHORT, "record has fewer words per shot than the circuit needs");
        max_n = std::max(max_n, p->n);
        const DevProg *dp = prog_desc(*p);
        for (uint32_t k = 0; k < G.shots; k++) {
            ResJob j{};
            j.prog = dp;
            j.st = to_dev(G.streams);
            j.record = (unsigned long long *)G.d_record;
            j.rec_stride = G.record_words;
            j.shot = k;
            hj.push_back({p->cost, j});
        }
        total += G.shots;
        if (G.shots) {
            cudaError_t e = cudaMemsetAsync(G.d_record, 0, (size_t)G.shots * G.record_words * 8, s);
            if (e) return cuda_fail(e, "clearing records");
        }
    }
    if (!total) return STAB_OK;
    // longest shots first (LPT order) for load balance
    std::stable_sort(hj.begin(), hj.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<ResJob> flat(hj.size());
    for (size_t i = 0; i < hj.size(); i++) flat[i] = hj[i].second;
    int rc = jobs.ensure(flat.size() * sizeof(ResJob));
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(jobs.p, flat.data(), flat.size() * sizeof(ResJob), cudaMemcpyHostToDevice, s);
    if (e) return cuda_fail(e, "uploading the job table");
    // the host vector must outlive the async copy
    e = cudaStreamSynchronize(s);
    if (e) return cuda_fail(e, "job table upload");
    stab_tune t = force ? *force : lookup_tune(ctx, max_n);
    e = resident_run((const ResJob *)jobs.p, (uint32_t)flat.size(), max_n, t, counter, ctx->d_err, ctx->lc, s,
                     &ctx->prof);
    if (e) return cuda_fail(e, "resident launch");
    return STAB_OK;
}

// Engine for `shots` shots of p.  The resident engine runs one shot per
// thread group for the whole circuit, so it needs many shots to fill the GPU
// and its time per shot grows quickly with n; the layered engine spreads each
// layer over 32-row slices of every tableau.  Measured on GB300 (rotated
// surface codes, 128 and ~800 shots): resident is faster only for tableaux of
// at most about 24 KB (d <= 9) given several hundred shots, or single-word
// tableaux (n <= 32).
bool prefer_resident(const stab_ctx *ctx, uint32_t n, uint64_t shots) {
    if (!resident_supported(n, ctx->lc)) return false;
    if (!layered_supported(n, ctx->lc)) return true;
    if ((n + 31) / 32 == 1) return true;
    return resident_smem_per_tableau(n) <= (24u << 10) && shots >= 512;
}

static uint32_t pick_engine(const stab_ctx *ctx, const HostProg &p, uint32_t engine, uint32_t shots) {
    if (engine != STAB_ENGINE_AUTO) return engine;
    return prefer_resident(ctx, p.n, shots) ? STAB_ENGINE_RESIDENT : STAB_ENGINE_LAYERED;
}

// Copy-bandwidth probe: `passes` passes of dst[i] = src[i] over n 16-byte
// words in one launch, loads and stores through L2 only (ld/st .cg), each
// thread keeping the same words on every pass.  With the two buffers smaller
// than L2 every pass after the first hits L2, so the launch measures L2
// read + write bandwidth without launch gaps between passes.
__global__ void __launch_bounds__(512) k_probe_copy(const uint4 *src, uint4 *dst, size_t n, uint32_t passes) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (uint32_t p = 0; p < passes; p++)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (i + k * stride < n) v[k] = __ldcg(src + i + k * stride);
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (i + k * stride < n) __stcg(dst + i + k * stride, v[k]);
        }
}

}  // namespace stab

using namespace stab;

#define CTX_GUARD                                                   \
    if (!ctx) return fail(STAB_ERR_ARG, "context is NULL");         \
    std::lock_guard<std::mutex> _lk(ctx->mu);                       \
    cudaSetDevice(ctx->device)

extern "C" {

const char *stab_last_error(void) { return g_err.c_str(); }

int stab_create(stab_ctx **out, int device, void *cuda_stream) {
    if (!out) return fail(STAB_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(STAB_ERR_ARG, "no such device");
    e = cudaSetDevice(device);
    if (e) return cuda_fail(e, "cudaSetDevice");
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e) return cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major < 10) return fail(STAB_ERR_UNSUPPORTED, "this build targets sm_103a (Blackwell)");
    auto *ctx = new stab_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->lc.sm_count = prop.multiProcessorCount;
    ctx->lc.smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaMalloc(&ctx->d_err, 512) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return fail(STAB_ERR_OOM, "cudaMalloc for the error flag failed");
    }
    ctx->d_counter = (unsigned int *)((char *)ctx->d_err + 128);
    ctx->d_stats = (unsigned long long *)((char *)ctx->d_err + 256);
    cudaMemset(ctx->d_err, 0, 512);
    if (const char *env = getenv("STAB_WAVE_CAPS")) {
        WaveCaps c;
        unsigned v[5];
        unsigned w6 = 0, w7 = 0;
        const int got = sscanf(env, "%u,%u,%u,%u,%u,%u,%u", &v[0], &v[1], &v[2], &v[3], &v[4], &w6, &w7);
        if (got >= 5) {
            c.pcap = v[0]; c.wcap = v[1]; c.paircap = v[2]; c.jcap = v[3]; c.mark_budget = v[4];
            if (got >= 6) c.window = w6;
            if (got >= 7) c.wave_limit = w7;
            set_wave_caps(c);
        }
    }
    *out = ctx;
    return STAB_OK;
}

int stab_serve_stop(stab_ctx *ctx);

void stab_destroy(stab_ctx *ctx) {
    if (!ctx) return;
    if (ctx->serve) stab_serve_stop(ctx);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        for (auto &kv : ctx->progs)
            free_prog(*kv.second);
        if (ctx->gslot.gs) cudaStreamSynchronize(ctx->gslot.gs);
        graph_slot_free(ctx->gslot);
        batch_free(ctx->resident);
        batch_free(ctx->tmp);
        ctx->ms_buf.release();
        ctx->jobs_buf.release();
        ctx->stage_coins.release();
        ctx->stage_noise.release();
        ctx->stage_rec.release();
        ctx->prof.collect();
        for (auto e : ctx->prof.pool) cudaEventDestroy(e);
        if (ctx->d_err) cudaFree(ctx->d_err);
    }
    delete ctx;
}

int stab_set_stream(stab_ctx *ctx, void *cuda_stream) {
    CTX_GUARD;
    ctx->stream = (cudaStream_t)cuda_stream;
    return STAB_OK;
}

int stab_sync(stab_ctx *ctx) {
    CTX_GUARD;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e) return cuda_fail(e, "stream synchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "reading the device error flag");
    if (flag) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        const char *what = flag == DERR_ODD_PHASE ? "odd power of i in a stabilizer product"
                         : flag == DERR_BAD_PRODUCT ? "deterministic product is not +-Z_a"
                         : flag == DERR_TIMEOUT ? "bounded device wait expired"
                         : "device bounds check failed";
        return fail(flag == DERR_TIMEOUT ? STAB_ERR_TIMEOUT : STAB_ERR_INTERNAL,
                    std::string("device consistency check: ") + what);
    }
    return STAB_OK;
}

int stab_compile(stab_ctx *ctx, uint32_t n, const stab_op *ops, size_t n_ops, const double *params,
                 size_t n_params, uint64_t *circuit_id) {
    CTX_GUARD;
    if (!circuit_id) return fail(STAB_ERR_ARG, "circuit_id is NULL");
    auto P = std::make_unique<HostProg>();
    std::string err;
    int rc = compile_program(n, ops, n_ops, params, n_params, *P, &err);
    if (rc) return fail(rc, err);
    rc = upload_prog(*P);
    if (rc) return rc;
    P->id = ctx->next_id++;
    *circuit_id = P->id;
    ctx->progs[P->id] = std::move(P);
    return STAB_OK;
}

int stab_circuit_info_get(stab_ctx *ctx, uint64_t circuit_id, stab_circuit_info *out) {
    CTX_GUARD;
    const HostProg *p = find_prog(ctx, circuit_id);
    if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id");
    if (!out) return fail(STAB_ERR_ARG, "out is NULL");
    *out = p->info;
    return STAB_OK;
}

int stab_compile_info(uint32_t n, const stab_op *ops, size_t n_ops, const double *params,
                      size_t n_params, stab_circuit_info *out) {
    if (!out) return fail(STAB_ERR_ARG, "out is NULL");
    HostProg P;                 // host vectors only: nothing reaches the device
    std::string err;
    const int rc = compile_program(n, ops, n_ops, params, n_params, P, &err);
    if (rc) return fail(rc, err);
    *out = P.info;
    return STAB_OK;
}

int stab_release_circuit(stab_ctx *ctx, uint64_t circuit_id) {
    CTX_GUARD;
    auto it = ctx->progs.find(circuit_id);
    if (it == ctx->progs.end()) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id");
    cudaStreamSynchronize(ctx->stream);
    free_prog(*it->second);
    ctx->progs.erase(it);
    return STAB_OK;
}

int stab_tableau_init(stab_ctx *ctx, uint32_t n, uint32_t count) {
    CTX_GUARD;
    if (n == 0 || count == 0) return fail(STAB_ERR_ARG, "n and count must be positive");
    if (count > 65535) return fail(STAB_ERR_UNSUPPORTED, "at most 65535 resident tableaux");
    if (!layered_supported(n, ctx->lc))
        return fail(STAB_ERR_UNSUPPORTED, "n = " + std::to_string(n) + " exceeds the layered engine's shared-memory slice");
    std::string err;
    cudaStreamSynchronize(ctx->stream);
    int rc = batch_alloc(ctx->resident, n, count, &err);
    if (rc) return fail(rc, err);
    cudaError_t e = layered_init(ctx->resident, ctx->stream, &ctx->prof);
    if (e) return cuda_fail(e, "tableau init");
    return STAB_OK;
}

int stab_apply_circuit(stab_ctx *ctx, uint64_t circuit_id, const stab_streams *streams,
                       uint64_t *d_record, uint64_t record_words) {
    CTX_GUARD;
    const HostProg *p = find_prog(ctx, circuit_id);
    if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id");
    Batch &b = ctx->resident;
    if (!b.count) return fail(STAB_ERR_ARG, "no resident tableaux: call stab_tableau_init first");
    if (b.n != p->n) return fail(STAB_ERR_ARG, "circuit qubit count differs from the resident tableaux");
    int rc = check_streams(*p, streams, b.count);
    if (rc) return rc;
    if (!d_record) return fail(STAB_ERR_ARG, "record buffer is NULL");
    if (record_words < p->info.record_words) return fail(STAB_ERR_STREAM_SHORT, "record buffer too short");
    rc = ensure_ms(ctx->ms, ctx->ms_buf, layered_prog(*p), b.count);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(d_record, 0, (size_t)b.count * record_words * 8, ctx->stream);
    if (e) return cuda_fail(e, "clearing records");
    GraphSlot *gsl = graph_slot_init(ctx->gslot) == 0 ? &ctx->gslot : nullptr;
    e = layered_run(layered_prog(*p), b, ctx->ms, to_dev(*streams), (unsigned long long *)d_record, record_words,
                    ctx->d_err, ctx->lc, ctx->stream, &ctx->prof, ctx->d_stats, gsl);
    if (e) return cuda_fail(e, "apply_circuit");
    return STAB_OK;
}

int stab_get_tableau(stab_ctx *ctx, uint32_t index, uint64_t *hx, uint64_t *hz, uint8_t *hr) {
    CTX_GUARD;
    Batch &b = ctx->resident;
    if (index >= b.count) return fail(STAB_ERR_ARG, "tableau index out of range");
    if (!hx || !hz || !hr) return fail(STAB_ERR_ARG, "host buffers are NULL");
    cudaError_t e = layered_sync_qm(b, ctx->stream);
    if (e) return cuda_fail(e, "syncing the column-packed copy");
    const uint32_t n = b.n, H = b.H, CW = b.CW, W = (n + 63) / 64;
    std::vector<uint32_t> q(b.qm_stride), r(CW);
    e = cudaMemcpyAsync(q.data(), b.qm + (size_t)index * b.qm_stride, 4 * b.qm_stride, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaMemcpyAsync(r.data(), b.r + (size_t)index * CW, 4 * CW, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) return cuda_fail(e, "copying the tableau");
    memset(hx, 0, sizeof(uint64_t) * 2 * n * W);
    memset(hz, 0, sizeof(uint64_t) * 2 * n * W);
    const uint32_t *qx = q.data(), *qz = qx + (size_t)CW * n;
    for (uint32_t row = 0; row < 2 * n; row++) {
        const uint32_t slot = row < n ? row : 32 * H + (row - n);
        const uint32_t w = slot >> 5, sh = slot & 31;
        uint64_t *xr = hx + (size_t)row * W, *zr = hz + (size_t)row * W;
        for (uint32_t j = 0; j < n; j++) {
            xr[j >> 6] |= (uint64_t)((qx[(size_t)w * n + j] >> sh) & 1u) << (j & 63);
            zr[j >> 6] |= (uint64_t)((qz[(size_t)w * n + j] >> sh) & 1u) << (j & 63);
        }
        hr[row] = (uint8_t)((r[w] >> sh) & 1u);
    }
    return STAB_OK;
}

int stab_commute(stab_ctx *ctx, uint32_t index, const uint64_t *d_px, const uint64_t *d_pz, size_t m,
                 uint64_t *d_out) {
    CTX_GUARD;
    Batch &b = ctx->resident;
    if (!b.count) return fail(STAB_ERR_ARG, "no resident tableaux: call stab_tableau_init first");
    if (index >= b.count) return fail(STAB_ERR_ARG, "tableau index out of range");
    if (!m) return STAB_OK;
    if (!d_px || !d_pz || !d_out) return fail(STAB_ERR_ARG, "Pauli or output buffer is NULL");
    cudaError_t e = layered_commute(b, index, (const unsigned long long *)d_px, (const unsigned long long *)d_pz, m,
                                    (unsigned long long *)d_out, ctx->stream, &ctx->prof);
    if (e) return cuda_fail(e, "commutation kernel");
    return STAB_OK;
}

int stab_set_tableau(stab_ctx *ctx, uint32_t index, const uint64_t *hx, const uint64_t *hz, const uint8_t *hr) {
    CTX_GUARD;
    Batch &b = ctx->resident;
    if (index >= b.count) return fail(STAB_ERR_ARG, "tableau index out of range");
    if (!hx || !hz || !hr) return fail(STAB_ERR_ARG, "host buffers are NULL");
    cudaError_t e = layered_sync_qm(b, ctx->stream);
    if (e) return cuda_fail(e, "syncing the column-packed copy");
    const uint32_t n = b.n, H = b.H, CW = b.CW, W = (n + 63) / 64;
    std::vector<uint32_t> q(b.qm_stride, 0u), r(CW, 0u);
    uint32_t *qx = q.data(), *qz = qx + (size_t)CW * n;
    for (uint32_t row = 0; row < 2 * n; row++) {
        const uint32_t slot = row < n ? row : 32 * H + (row - n);
        const uint32_t w = slot >> 5, sh = slot & 31;
        const uint64_t *xr = hx + (size_t)row * W, *zr = hz + (size_t)row * W;
        for (uint32_t j = 0; j < n; j++) {
            qx[(size_t)w * n + j] |= (uint32_t)((xr[j >> 6] >> (j & 63)) & 1u) << sh;
            qz[(size_t)w * n + j] |= (uint32_t)((zr[j >> 6] >> (j & 63)) & 1u) << sh;
        }
        r[w] |= (uint32_t)(hr[row] & 1u) << sh;
    }
    e = cudaMemcpyAsync(b.qm + (size_t)index * b.qm_stride, q.data(), 4 * b.qm_stride, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaMemcpyAsync(b.r + (size_t)index * CW, r.data(), 4 * CW, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) return cuda_fail(e, "uploading the tableau");
    b.rm_valid = false;       // the next measurement layer rebuilds the row-packed copy
    return STAB_OK;
}

int stab_sample(stab_ctx *ctx, uint64_t circuit_id, uint32_t shots, const stab_streams *streams,
                uint64_t *d_record, uint64_t record_words, uint32_t engine) {
    CTX_GUARD;
    const HostProg *p = find_prog(ctx, circuit_id);
    if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id");
    int rc = check_streams(*p, streams, shots);
    if (rc) return rc;
    if (shots == 0) return STAB_OK;
    if (!d_record) return fail(STAB_ERR_ARG, "record buffer is NULL");
    if (record_words < p->info.record_words) return fail(STAB_ERR_STREAM_SHORT, "record buffer too short");
    const uint32_t eng = pick_engine(ctx, *p, engine, shots);
    if (eng == STAB_ENGINE_RESIDENT) {
        stab_job_group g{};
        g.circuit_id = circuit_id;
        g.shots = shots;
        g.streams = *streams;
        g.d_record = d_record;
        g.record_words = record_words;
        return run_resident_groups(ctx, &g, 1, nullptr, ctx->stream, ctx->jobs_buf, ctx->d_counter);
    }
    if (eng != STAB_ENGINE_LAYERED) return fail(STAB_ERR_ARG, "unknown engine");
    cudaError_t e = cudaMemsetAsync(d_record, 0, (size_t)shots * record_words * 8, ctx->stream);
    if (e) return cuda_fail(e, "clearing records");
    return run_layered_shots(ctx, *p, shots, *streams, d_record, record_words, ctx->stream, ctx->tmp,
                             ctx->ms, ctx->ms_buf);
}

int stab_sample_host(stab_ctx *ctx, uint64_t circuit_id, uint32_t shots, const uint64_t *host_coins,
                     uint64_t coin_words, const uint32_t *host_noise, uint64_t noise_words,
                     uint64_t *host_record, uint64_t record_words, uint32_t engine) {
    stab_streams st{};
    uint64_t *d_rec = nullptr;
    {
        CTX_GUARD;
        const HostProg *p = find_prog(ctx, circuit_id);
        if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id");
        if (!host_record) return fail(STAB_ERR_ARG, "host record is NULL");
        st.mode = STAB_STREAM_BUFFER;
        const size_t cb = (size_t)shots * coin_words * 8, nb = (size_t)shots * noise_words * 4;
        int rc = ctx->stage_coins.ensure(std::max<size_t>(cb, 8));
        if (!rc) rc = ctx->stage_noise.ensure(std::max<size_t>(nb, 8));
        if (!rc) rc = ctx->stage_rec.ensure(std::max<size_t>((size_t)shots * record_words * 8, 8));
        if (rc) return rc;
        cudaError_t e = cudaSuccess;
        if (cb && host_coins) e = cudaMemcpyAsync(ctx->stage_coins.p, host_coins, cb, cudaMemcpyHostToDevice, ctx->stream);
        if (!e && nb && host_noise) e = cudaMemcpyAsync(ctx->stage_noise.p, host_noise, nb, cudaMemcpyHostToDevice, ctx->stream);
        if (e) return cuda_fail(e, "copying streams to the device");
        st.coins = host_coins ? (const uint64_t *)ctx->stage_coins.p : nullptr;
        st.coin_words = coin_words;
        st.noise = host_noise ? (const uint32_t *)ctx->stage_noise.p : nullptr;
        st.noise_words = noise_words;
        d_rec = (uint64_t *)ctx->stage_rec.p;
    }
    int rc = stab_sample(ctx, circuit_id, shots, &st, d_rec, record_words, engine);
    if (rc) return rc;
    CTX_GUARD;
    cudaError_t e = cudaMemcpyAsync(host_record, d_rec, (size_t)shots * record_words * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) return cuda_fail(e, "copying records to the host");
    return STAB_OK;
}

int stab_sample_batch(stab_ctx *ctx, const stab_job_group *groups, size_t n_groups) {
    CTX_GUARD;
    if (n_groups && !groups) return fail(STAB_ERR_ARG, "groups is NULL");
    // Groups of small tableaux share one persistent resident-engine launch;
    // groups whose tableaux are too large for it to win run through the
    // layered engine afterwards (the resident launch fills every SM, so the
    // two would not overlap anyway).
    uint64_t total = 0;
    for (size_t gi = 0; gi < n_groups; gi++) total += groups[gi].shots;
    std::vector<stab_job_group> res, lay;
    for (size_t gi = 0; gi < n_groups; gi++) {
        const HostProg *p = find_prog(ctx, groups[gi].circuit_id);
        if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id " + std::to_string(groups[gi].circuit_id));
        if (prefer_resident(ctx, p->n, total)) res.push_back(groups[gi]);
        else lay.push_back(groups[gi]);
    }
    // validate every layered group before launching anything
    for (const stab_job_group &G : lay) {
        const HostProg *p = find_prog(ctx, G.circuit_id);
        int rc = check_streams(*p, &G.streams, G.shots);
        if (rc) return rc;
        if (G.shots && !G.d_record) return fail(STAB_ERR_ARG, "record buffer is NULL");
        if (G.record_words < p->info.record_words)
            return fail(STAB_ERR_STREAM_SHORT, "record has fewer words per shot than the circuit needs");
    }
    int rc = run_resident_groups(ctx, res.data(), res.size(), nullptr, ctx->stream, ctx->jobs_buf, ctx->d_counter);
    if (rc) return rc;
    for (const stab_job_group &G : lay) {
        if (!G.shots) continue;
        const HostProg *p = find_prog(ctx, G.circuit_id);
        cudaError_t e = cudaMemsetAsync(G.d_record, 0, (size_t)G.shots * G.record_words * 8, ctx->stream);
        if (e) return cuda_fail(e, "clearing records");
        rc = run_layered_shots(ctx, *p, G.shots, G.streams, G.d_record, G.record_words, ctx->stream, ctx->tmp,
                               ctx->ms, ctx->ms_buf);
        if (rc) return rc;
    }
    return STAB_OK;
}

int stab_get_tune(stab_ctx *ctx, uint32_t n, stab_tune *out) {
    CTX_GUARD;
    if (!out) return fail(STAB_ERR_ARG, "out is NULL");
    *out = lookup_tune(ctx, n);
    return STAB_OK;
}

int stab_set_tune(stab_ctx *ctx, uint32_t n, const stab_tune *t) {
    CTX_GUARD;
    if (!t) return fail(STAB_ERR_ARG, "tune is NULL");
    const uint32_t G = t->group_threads, tpc = t->tableaux_per_cta, wpt = t->words_per_thread;
    if (!(G == 32 || G == 64 || G == 128 || G == 256) || tpc < 1 || G * tpc > 1024 ||
        (G > 32 && tpc > 15) || !(wpt == 1 || wpt == 2 || wpt == 4) || !resident_shape_ok(n, *t, ctx->lc))
        return fail(STAB_ERR_ARG, "invalid resident launch shape");
    if (resident_smem_per_tableau(n) * tpc > ctx->lc.smem_optin)
        return fail(STAB_ERR_ARG, "shape needs more shared memory than a CTA has");
    ctx->tune[(n + 31) / 32] = *t;
    return STAB_OK;
}

int stab_autotune(stab_ctx *ctx, const uint64_t *circuit_ids, size_t n_circuits, uint32_t shots) {
    CTX_GUARD;
    if (!circuit_ids && n_circuits) return fail(STAB_ERR_ARG, "circuit_ids is NULL");
    DevBuf rec;
    for (size_t ci = 0; ci < n_circuits; ci++) {
        const HostProg *p = find_prog(ctx, circuit_ids[ci]);
        if (!p) return fail(STAB_ERR_NOT_FOUND, "unknown circuit id");
        if (!resident_supported(p->n, ctx->lc)) continue;
        int rc = rec.ensure((size_t)shots * p->info.record_words * 8);
        if (rc) return rc;
        stab_job_group g{};
        g.circuit_id = p->id;
        g.shots = shots;
        g.streams.mode = STAB_STREAM_SEEDED;
        g.streams.seed = 12345;
        g.d_record = (uint64_t *)rec.p;
        g.record_words = p->info.record_words;
        float best = 1e30f;
        stab_tune best_t = default_tune(ctx, p->n);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const size_t per = resident_smem_per_tableau(p->n);
        for (uint32_t G : {32u, 64u, 128u, 256u})
            for (uint32_t tpc : {1u, 2u, 4u, 8u})
                for (uint32_t wpt : {1u, 2u, 4u}) {
                    if (G * tpc > 1024 || (G > 32 && tpc > 15) || per * tpc > ctx->lc.smem_optin) continue;
                    if (wpt > p->CW) continue;
                    stab_tune t{G, tpc, wpt, 0};
                    if (!resident_shape_ok(p->n, t, ctx->lc)) continue;
                    // one warm-up, then time
                    int rc2 = run_resident_groups(ctx, &g, 1, &t, ctx->stream, ctx->jobs_buf, ctx->d_counter);
                    if (rc2) { rec.release(); return rc2; }
                    cudaEventRecord(e0, ctx->stream);
                    rc2 = run_resident_groups(ctx, &g, 1, &t, ctx->stream, ctx->jobs_buf, ctx->d_counter);
                    if (rc2) { rec.release(); return rc2; }
                    cudaEventRecord(e1, ctx->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) { best = ms; best_t = t; }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->tune[(p->n + 31) / 32] = best_t;
    }
    cudaStreamSynchronize(ctx->stream);
    rec.release();
    return STAB_OK;
}

int stab_profile(stab_ctx *ctx, uint32_t kind_mask) {
    CTX_GUARD;
    ctx->prof.mask = kind_mask;
    return STAB_OK;
}

int stab_profile_read(stab_ctx *ctx, uint32_t kind, stab_kernel_stats *out, int reset) {
    CTX_GUARD;
    if (!out || kind >= STAB_N_KERNEL_KINDS) return fail(STAB_ERR_ARG, "bad profile_read arguments");
    int rc = ctx->prof.collect();
    if (rc) return rc;
    out->launches = ctx->prof.n[kind];
    out->total_ms = ctx->prof.ms[kind];
    out->alg_bytes = ctx->prof.bytes[kind];
    if (reset) {
        ctx->prof.n[kind] = 0;
        ctx->prof.ms[kind] = 0.0;
        ctx->prof.bytes[kind] = 0.0;
    }
    return STAB_OK;
}

int stab_launch_count(stab_ctx *ctx, uint64_t *count, int reset) {
    CTX_GUARD;
    if (!count) return fail(STAB_ERR_ARG, "count is NULL");
    *count = ctx->prof.launches;
    if (reset) ctx->prof.launches = 0;
    return STAB_OK;
}

int stab_probe_copy(stab_ctx *ctx, uint64_t bytes, uint32_t passes, double *gbs) {
    CTX_GUARD;
    if (!gbs || passes == 0 || bytes < 4096) return fail(STAB_ERR_ARG, "bad probe arguments");
    const size_t half = (size_t)(bytes / 2) & ~(size_t)15;
    void *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, half) != cudaSuccess || cudaMalloc(&b, half) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaFree(a);
        return fail(STAB_ERR_OOM, "cudaMalloc for the probe buffers failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(a, 1, half, ctx->stream);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    const uint32_t grid = 4u * (uint32_t)ctx->lc.sm_count;
    const size_t n = half / 16;
    float ms = 0.f;
    if (!e) {
        k_probe_copy<<<grid, 512, 0, ctx->stream>>>((const uint4 *)a, (uint4 *)b, n, 1);   // warm-up pass
        cudaEventRecord(e0, ctx->stream);
        k_probe_copy<<<grid, 512, 0, ctx->stream>>>((const uint4 *)a, (uint4 *)b, n, passes);
        cudaEventRecord(e1, ctx->stream);
        e = cudaEventSynchronize(e1);
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    if (e) return cuda_fail(e, "copy probe");
    *gbs = 2.0 * (double)(n * 16) * passes / (ms * 1e-3) / 1e9;
    return STAB_OK;
}

int stab_engine_counters(stab_ctx *ctx, uint64_t *out, size_t n, int reset) {
    CTX_GUARD;
    if (!out || n == 0) return fail(STAB_ERR_ARG, "bad counter buffer");
    unsigned long long v[DC_N];
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (!e) e = cudaMemcpy(v, ctx->d_stats, sizeof(v), cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "reading engine counters");
    for (size_t i = 0; i < n && i < (size_t)DC_N; i++) out[i] = v[i];
    if (reset) cudaMemset(ctx->d_stats, 0, sizeof(v));
    return STAB_OK;
}

}  // extern "C"
