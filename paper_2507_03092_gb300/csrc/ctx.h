// ctx.h -- the context object behind stab_ctx* (host side, not ABI).
#pragma once
#include "internal.h"

#include <atomic>
#include <condition_variable>
#include <deque>
#include <thread>

namespace stab {

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

struct DevBuf {                 // grow-only device buffer
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes);
    void release();
};

struct ServeState;              // serve.cpp

}  // namespace stab

struct stab_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    stab::LaunchCfg lc;
    std::mutex mu;                                   // guards everything below
    std::map<uint64_t, std::unique_ptr<stab::HostProg>> progs;
    uint64_t next_id = 1;
    stab::Batch resident;                            // tableau_init / apply_circuit
    stab::Batch tmp;                                 // layered sample workspace
    stab::MeasScratch ms;
    stab::DevBuf ms_buf, jobs_buf, stage_coins, stage_noise, stage_rec;
    int *d_err = nullptr;
    unsigned int *d_counter = nullptr;
    unsigned long long *d_stats = nullptr;          // DC_* counters
    std::map<uint32_t, stab_tune> tune;              // bucket ceil(n/32) -> shape
    stab::KernelProf prof;
    stab::GraphSlot gslot;                          // graph replay for work on `stream`
    stab::ServeState *serve = nullptr;
};

namespace stab {
stab_tune default_tune(const stab_ctx *ctx, uint32_t n);
stab_tune lookup_tune(const stab_ctx *ctx, uint32_t n);
const HostProg *find_prog(stab_ctx *ctx, uint64_t id);
// engine choice from measured per-shot costs (AUTO and serving)
bool prefer_resident(const stab_ctx *ctx, uint32_t n, uint64_t shots);
const DevProg *prog_desc(const HostProg &p);     // device copy of p's descriptor
DevStreams to_dev(const stab_streams &s);
int check_streams(const HostProg &p, const stab_streams *s, uint32_t shots);
// launch the resident engine over job groups (ctx->mu held)
int run_resident_groups(stab_ctx *ctx, const stab_job_group *groups, size_t n_groups,
                        const stab_tune *force, cudaStream_t s, DevBuf &jobs, unsigned int *counter);
int run_layered_shots(stab_ctx *ctx, const HostProg &p, uint32_t shots, const stab_streams &st,
                      uint64_t *d_record, uint64_t record_words, cudaStream_t s, Batch &work,
                      MeasScratch &ms, DevBuf &ms_buf);
}  // namespace stab
