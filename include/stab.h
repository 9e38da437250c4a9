/*
 * stab.h -- C ABI of libstab.so, a GB300 (sm_103a) CHP stabilizer-tableau
 * simulator (arXiv 2507.03092, "STABSim", hot path).
 *
 * All arithmetic is exact GF(2) / mod-4 integer work.  Every entry point
 * returns STAB_OK (0) or a negative STAB_ERR_* code; nothing is thrown across
 * the ABI.  stab_last_error() returns a thread-local message for the last
 * failing call on the calling thread.  Host-side validation (qubit indices,
 * distinct 2-qubit operands, stream lengths, sizes) happens before any launch.
 *
 * Ownership: buffers passed in are owned by the caller (device buffers are
 * typically torch tensors); the library owns only its contexts, compiled
 * circuits and tableau storage.  Launches are asynchronous on the context's
 * CUDA stream and stream-ordered with the caller's work on that stream;
 * stab_sync() waits for them and reports device-side error flags.
 *
 * Conventions shared with the CPU oracle (each side implements them itself):
 *  - Tableau (Sec. 2.3, "The CHP Formalism"): 2n rows, rows 0..n-1
 *    destabilizers, n..2n-1 stabilizers, each x[0..n), z[0..n) and sign r.
 *    Initial state |0...0>: destabilizer i = X_i, stabilizer i = Z_i.
 *  - Coins: the m-th M/R/MPP op (circuit order) reads bit m%64 of coin word m/64
 *    of its shot, and only if its outcome is random (Sec. 2.4: "a random phase
 *    bit ... is chosen").  Outcome 1 means eigenvalue -1.
 *  - Records: bit k of a shot's record is the outcome of the k-th M or MPP op.
 *  - MPP (Pauli-product measurement): measures the product P of its factors'
 *    Pauli matrices; outcome 1 = eigenvalue -1; one coin slot, like M.  A
 *    random outcome makes (-1)^coin P the new stabilizer (Sec. 2.4's update
 *    with Z_a replaced by P; commutation of a row with P as in Sec. 3.2).
 *  - Noise: the l-th noise op reads uint32 word l of its shot's noise stream
 *    (RESET_ERROR reads words l, l+1, l+2).  T(p) = floor(p * 2^32).
 *    DEPOLARIZE1(p): error iff u < T, Pauli (u*3)/T = X, Y, Z.
 *    DEPOLARIZE2(p): error iff u < T, m = (u*15)/T + 1, Pauli m/4 on q0 and
 *    m%4 on q1 (0 I, 1 X, 2 Y, 3 Z).  PAULI_CHANNEL_1(px,py,pz): X if
 *    u < T(px), Y if u < T(px)+T(py), Z if u < T(px)+T(py)+T(pz).
 *    RESET_ERROR(gamma, q): if u0 < T(gamma) reset the qubit with coin u1&1,
 *    then Z if u2 < T(q) (composite relaxation/dephasing, Sec. 4.2).
 *  - SEEDED streams: coin word k of shot s = SplitMix64 output k of
 *    key(seed, s, 1); noise word l = (output l of key(seed, s, 2)) >> 32, where
 *    key(seed, s, kind) = mix64(mix64(seed + kind*G) + (s+1)*G), G the
 *    SplitMix64 increment (Steele, Lea & Flood 2014).
 */
#ifndef LIBSTAB_STAB_H_
#define LIBSTAB_STAB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define STAB_OK 0
#define STAB_ERR_ARG (-1)          /* invalid argument (index, size, pointer) */
#define STAB_ERR_OOM (-2)          /* device or host allocation failed / footprint too large */
#define STAB_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define STAB_ERR_STREAM_SHORT (-4) /* a coin/noise/record buffer is shorter than the circuit needs */
#define STAB_ERR_TIMEOUT (-5)      /* a bounded wait gave up (device flag or host poll) */
#define STAB_ERR_BUSY (-6)         /* the request queue or slot table is full */
#define STAB_ERR_INTERNAL (-7)     /* a device-side consistency check failed (odd phase, bad product) */
#define STAB_ERR_NOT_FOUND (-8)    /* unknown circuit or request id */
#define STAB_ERR_UNSUPPORTED (-9)  /* size outside what the chosen engine supports */

/* ---- op kinds (values are part of the ABI) ---- */
enum stab_kind {
    STAB_NOP = 0,
    STAB_H = 1, STAB_S = 2, STAB_X = 3, STAB_Y = 4, STAB_Z = 5, /* one-qubit Cliffords, Sec. 2.4 Table */
    STAB_CX = 6,      /* q0 control, q1 target */
    STAB_CZ = 7, STAB_SWAP = 8,
    STAB_M = 9,       /* Z-basis measurement, recorded */
    STAB_R = 10,      /* reset to |0>: measure (not recorded), then X if the outcome is 1 */
    STAB_DEP1 = 11,   /* DEPOLARIZE1(p): params[arg] = (p, -, -) */
    STAB_DEP2 = 12,   /* DEPOLARIZE2(p) on (q0, q1): params[arg] = (p, -, -) */
    STAB_PC1 = 13,    /* PAULI_CHANNEL_1: params[arg] = (px, py, pz) */
    STAB_TICK = 14,   /* layer hint, no effect */
    STAB_RESET_ERR = 15, /* RESET_ERROR: params[arg] = (gamma, q, -) */
    STAB_MPP = 16,    /* Pauli-product measurement, recorded: q0 = number of factors k (1..64),
                         followed by k STAB_PAULI ops on distinct qubits */
    STAB_PAULI = 17   /* factor of the preceding MPP: q0 = qubit, q1 = 1 X, 2 Y, 3 Z */
};

/* One op: 16 bytes, little-endian, identical to the Python OP_DTYPE. */
typedef struct stab_op {
    uint8_t kind;
    uint8_t rsv0;
    uint16_t rsv1;
    uint32_t q0;
    uint32_t q1;
    uint32_t arg; /* noise ops: row index into the params table */
} stab_op;

/* ---- coin / noise streams ---- */
#define STAB_STREAM_BUFFER 0u /* caller-provided device buffers, one row per shot */
#define STAB_STREAM_SEEDED 1u /* generated on the device from (seed, shot_offset + shot) */

typedef struct stab_streams {
    uint32_t mode;
    uint32_t rsv;
    uint64_t seed;          /* SEEDED */
    uint64_t shot_offset;   /* SEEDED: stream shot index of the call's first shot */
    const uint64_t *coins;  /* BUFFER: device pointer, [shots][coin_words] */
    uint64_t coin_words;    /* BUFFER: row stride in uint64 words */
    const uint32_t *noise;  /* BUFFER: device pointer, [shots][noise_words] */
    uint64_t noise_words;   /* BUFFER: row stride in uint32 words */
} stab_streams;

typedef struct stab_circuit_info {
    uint32_t n;              /* qubits */
    uint32_t n_layers;       /* compiled layers (gate layers + measurement layers) */
    uint64_t n_ops;          /* ops excluding NOP/TICK */
    uint64_t n_gates;        /* unitary gates */
    uint64_t n_meas;         /* M and MPP ops = record bits */
    uint64_t n_coin;         /* M, R and MPP ops = coin slots */
    uint64_t n_noise_words;  /* noise words one shot reads */
    uint64_t record_words;   /* ceil(n_meas / 64), at least 1 */
    uint64_t coin_words;     /* ceil(n_coin / 64), at least 1 */
    uint32_t n_gate_layers;
    uint32_t n_meas_layers;
    uint32_t n_gate_runs;    /* maximal runs of consecutive gate layers */
    uint32_t max_layer_meas; /* largest measurement layer */
} stab_circuit_info;

/* engines for stab_sample */
#define STAB_ENGINE_AUTO 0u      /* resident for tableaux of <= 24 KB (n <= ~200) with >= 512 shots
                                   or n <= 32, layered otherwise (from measured per-shot costs) */
#define STAB_ENGINE_LAYERED 1u  /* tableau in HBM/L2, one launch per gate run / measurement layer */
#define STAB_ENGINE_RESIDENT 2u /* tableau in shared memory, whole circuit in one persistent launch */

typedef struct stab_ctx stab_ctx;

/* Context bound to CUDA device `device`; `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream), e.g. torch.cuda.current_stream().cuda_stream. */
int stab_create(stab_ctx **out, int device, void *cuda_stream);
void stab_destroy(stab_ctx *ctx);
int stab_set_stream(stab_ctx *ctx, void *cuda_stream);
const char *stab_last_error(void);
/* Wait for the context's stream; returns a device-side error flag if one was set. */
int stab_sync(stab_ctx *ctx);

/* Compile a flat op list (host memory, copied) over n qubits into layers of
 * pairwise-disjoint ops (the paper's sim2d chunking done at generation time,
 * Sec. 3.1.4).  params: host float64 [n_params][3]. */
int stab_compile(stab_ctx *ctx, uint32_t n, const stab_op *ops, size_t n_ops,
                 const double *params, size_t n_params, uint64_t *circuit_id);
int stab_circuit_info_get(stab_ctx *ctx, uint64_t circuit_id, stab_circuit_info *out);
/* Validate and compile a flat op list on the host only -- no context, no
 * device, nothing kept -- and return what stab_compile would report for it
 * (layer counts, record, coin and noise sizes).  Arguments and errors as for
 * stab_compile; *out is written only on success. */
int stab_compile_info(uint32_t n, const stab_op *ops, size_t n_ops, const double *params,
                      size_t n_params, stab_circuit_info *out);
int stab_release_circuit(stab_ctx *ctx, uint64_t circuit_id);

/* ---- resident tableaux: tableau_init(n), apply_circuit(...) ---- */

/* (Re)allocate `count` resident tableaux of n qubits on the device, each |0...0>
 * (Sec. 2.3; 4n^2+2n bits each, stored twice: column-packed and row-packed). */
int stab_tableau_init(stab_ctx *ctx, uint32_t n, uint32_t count);
/* Evolve every resident tableau i through the circuit (tableau i reads stream
 * row / shot i): the paper's sim(circuit) (Sec. 3.1.4, Scheduling Experiment),
 * with its chunking of independent gates done at compile time; gates by the
 * Sec. 2.4 Table, measurement and reset by the Sec. 2.4 rules with Appendix B's
 * rowsum.  d_record: device [count][record_words] uint64, overwritten. */
int stab_apply_circuit(stab_ctx *ctx, uint64_t circuit_id, const stab_streams *streams,
                       uint64_t *d_record, uint64_t record_words);
/* Copy resident tableau `index` to host in the row-major form of Sec. 2.3 (The
 * CHP Formalism: rows 0..n-1 destabilizers, n..2n-1 stabilizers): x, z as
 * uint64 [2n][ceil(n/64)] (bit j of row i = qubit j), r as uint8 [2n].
 * Synchronizes.  stab_set_tableau writes one in the same layout (checkpoint /
 * restore); the caller is responsible for it being a valid tableau. */
int stab_get_tableau(stab_ctx *ctx, uint32_t index, uint64_t *host_x, uint64_t *host_z,
                     uint8_t *host_r);
int stab_set_tableau(stab_ctx *ctx, uint32_t index, const uint64_t *host_x,
                     const uint64_t *host_z, const uint8_t *host_r);

/* Commutation of m Pauli strings with every row of resident tableau `index`
 * (Sec. 3.2: row S anticommutes with P iff x_P . z_S + z_P . x_S is odd).
 *   d_px, d_pz: device uint64 [m][ceil(n/64)], bit j = the X / Z part of the
 *               Pauli on qubit j (X: x, Y: x and z, Z: z); bits >= n ignored.
 *   d_out:      device uint64 [m][2 ceil(n/64)], overwritten: words
 *               [0, ceil(n/64)) hold bit i = destabilizer i anticommutes, words
 *               [ceil(n/64), 2 ceil(n/64)) bit i = stabilizer i anticommutes.
 * Caller owns all buffers.  Asynchronous on the context's stream; m = 0 does
 * nothing.  Errors: STAB_ERR_ARG (no tableaux, index out of range, NULL
 * buffers with m > 0). */
int stab_commute(stab_ctx *ctx, uint32_t index, const uint64_t *d_px, const uint64_t *d_pz,
                 size_t m, uint64_t *d_out);

/* ---- sample(shots, streams) -> records: every shot from |0...0> ---- */

/* Shots of a circuit, each from |0...0> (Sec. 2.3 initial tableau) through
 * sim(circuit) (Sec. 3.1.4), random outcomes read from the coin stream (Sec.
 * 2.4: "a random phase bit ... is chosen") and Pauli errors injected from the
 * noise stream (Sec. 2.6, QEC operations; Sec. 2.7, stochastic Pauli
 * channels); the paper names sampling many shots in parallel on the GPU as
 * future work (Sec. 6).  Records, coins and noise as in the header comment.
 * d_record: device [shots][record_words] uint64, overwritten.  Asynchronous
 * on the context's stream.  On the layered engine the call's launch sequence
 * is captured once per (circuit, batch shape) into a CUDA graph, run on an
 * internal stream ordered after and before the context's stream by events,
 * and replayed on later calls (the streams and record pointer are copied to
 * device memory for each call, so the caller may reuse its stab_streams at
 * once); while per-launch profiling is on (stab_profile) the kernels are
 * launched one by one instead.  Engine choice for STAB_ENGINE_AUTO: see above. */
int stab_sample(stab_ctx *ctx, uint64_t circuit_id, uint32_t shots, const stab_streams *streams,
                uint64_t *d_record, uint64_t record_words, uint32_t engine);
/* Same with HOST buffers: copies coins/noise to the device, runs, copies the
 * records back, and synchronizes.  host_noise may be NULL for noiseless circuits.
 * Arguments as stab_sample's, with host_coins [shots][coin_words] uint64,
 * host_noise [shots][noise_words] uint32 and host_record [shots][record_words]
 * uint64 in host memory (pinned memory makes the copies faster).  Errors as
 * stab_sample's, plus STAB_ERR_OOM if the device staging buffers cannot grow. */
int stab_sample_host(stab_ctx *ctx, uint64_t circuit_id, uint32_t shots,
                     const uint64_t *host_coins, uint64_t coin_words,
                     const uint32_t *host_noise, uint64_t noise_words,
                     uint64_t *host_record, uint64_t record_words, uint32_t engine);

/* ---- batched form: many circuits (uneven sizes) in one persistent launch ---- */
typedef struct stab_job_group {
    uint64_t circuit_id;
    uint32_t shots;
    uint32_t rsv;
    stab_streams streams;
    uint64_t *d_record;     /* device [shots][record_words] */
    uint64_t record_words;
} stab_job_group;

/* Every shot of every group, records keyed by (group streams, shot index) as in
 * stab_sample.  Groups of small tableaux (the same rule as STAB_ENGINE_AUTO,
 * with the batch's total shot count) run together in one persistent
 * resident-engine launch shaped by the autotuner; the other groups then run
 * through the layered engine, one launch sequence per group.  Asynchronous on
 * the context's stream except for the job-table upload. */
int stab_sample_batch(stab_ctx *ctx, const stab_job_group *groups, size_t n_groups);

/* One persistent resident-engine launch like stab_sample_batch's (every group
 * on the resident engine), for callers that cannot allocate device memory at
 * call time: code running where every device allocation is owned by a host
 * framework's memory pool, or latency-critical loops that cannot afford
 * cudaMalloc's implicit synchronisation.  (The paper has no counterpart; this
 * is a property of this library.)  The resident engine's only global scratch,
 * its job table and work counter, live in a fixed array compiled into the
 * library instead of memory from cudaMalloc: at most 8192 shots in total and
 * 64 groups per call (about 0.7 MiB, held on every GPU that loads the library
 * until the process exits); larger batches are rejected with
 * STAB_ERR_UNSUPPORTED before anything is launched.  The call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library call): the job table
 * is written on the device by a small kernel from the call's group list,
 * passed by value as a kernel argument, so there is no host staging buffer.
 * The caller still passes the streams and record buffers, and the circuits
 * must have been compiled before.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current, so
 * make that first call before any stream capture.  Every call shares the
 * array: calls whose launches overlap on the GPU (for instance calls on two
 * contexts with different streams) race on it; each call clears the work
 * counter before its launch. */
int stab_sample_batch_noalloc(stab_ctx *ctx, const stab_job_group *groups, size_t n_groups);

/* Resident-engine launch shape, chosen per qubit-count bucket by the autotuner. */
typedef struct stab_tune {
    uint32_t group_threads;    /* threads per tableau: 32, 64, 128 or 256 */
    uint32_t tableaux_per_cta; /* tableaux resident per CTA */
    uint32_t words_per_thread; /* 32-bit tableau words per thread per gate item: 1, 2 or 4 */
    uint32_t rsv;
} stab_tune;

/* Time the candidate shapes on `shots` shots of each circuit and store the
 * fastest per bucket (bucket = ceil(n/32)).  Synchronizes. */
int stab_autotune(stab_ctx *ctx, const uint64_t *circuit_ids, size_t n_circuits, uint32_t shots);
int stab_get_tune(stab_ctx *ctx, uint32_t n, stab_tune *out);
int stab_set_tune(stab_ctx *ctx, uint32_t n, const stab_tune *tune);

/* ---- served form: continuous batching with HBM-footprint admission ----
 * The paper has no serving layer; this one runs the same per-shot simulation
 * as stab_sample (Sec. 2.3-2.4, Sec. 3.1.4) for requests that arrive over
 * time, toward the Sec. 6 direction of parallel sampling on the GPU.  Requests
 * are admitted in arrival order when a launch slot is free and their device
 * footprint fits hbm_budget_bytes; small-tableau requests waiting together
 * share one resident-engine launch, larger ones get a layered launch sequence,
 * and each launch runs on its own stream so admitted work overlaps.  A
 * request's records depend only on (circuit, seed, shot_offset), never on the
 * mix it was served in. */
typedef struct stab_serve_config {
    uint64_t hbm_budget_bytes; /* admission limit for resident request state */
    uint32_t max_inflight;     /* concurrently admitted requests (slots) */
    uint32_t n_streams;        /* device streams the loop spreads launches over */
    uint32_t max_batch_requests; /* small requests merged into one resident launch */
    uint32_t rsv;
} stab_serve_config;

typedef struct stab_request_status {
    uint64_t req_id;
    int32_t status;         /* STAB_OK or an error code */
    uint32_t shots;
    double t_submit;        /* seconds, CLOCK_MONOTONIC */
    double t_admit;
    double t_done;
} stab_request_status;

/* Start the request loop (one scheduler thread, n_streams device streams).
 * Errors: STAB_ERR_ARG (NULL or zero-sized config), STAB_ERR_BUSY (already
 * started), STAB_ERR_CUDA / STAB_ERR_OOM (stream or counter creation). */
int stab_serve_start(stab_ctx *ctx, const stab_serve_config *cfg);
/* Queue a request: `shots` shots of a compiled circuit with SEEDED streams
 * (seed, shot_offset); records land in d_record ([shots][record_words], device,
 * caller-owned, must stay valid until the request completes). */
int stab_serve_submit(stab_ctx *ctx, uint64_t circuit_id, uint32_t shots, uint64_t seed,
                      uint64_t shot_offset, uint64_t *d_record, uint64_t record_words,
                      uint64_t *req_id);
/* Collect up to `cap` completed requests (non-blocking); *n_done = number written. */
int stab_serve_poll(stab_ctx *ctx, stab_request_status *done, size_t cap, size_t *n_done);
/* Wait until every submitted request completed or `timeout_s` elapsed. */
int stab_serve_drain(stab_ctx *ctx, double timeout_s);
/* Stop the loop after the launches in flight finish; queued requests that were
 * never admitted are dropped.  Frees the loop's streams and device state. */
int stab_serve_stop(stab_ctx *ctx);

/* ---- instrumentation (benchmarks) ---- */
#define STAB_KERNEL_GATE_RUN 0u  /* layered engine: run of gate layers on one 32-row slice */
#define STAB_KERNEL_MEAS_DET 1u  /* layered engine: pivot test + deterministic outcomes */
#define STAB_KERNEL_MEAS_RAND 2u /* layered engine: random measurements of a layer */
#define STAB_KERNEL_OTHER 3u     /* layered engine: init, transposes, column gather, conditional Paulis */
#define STAB_KERNEL_RESIDENT 4u  /* resident engine persistent launch */
#define STAB_KERNEL_COMMUTE 5u   /* Pauli-vs-tableau commutation (stab_commute) */
#define STAB_N_KERNEL_KINDS 6u

typedef struct stab_kernel_stats {
    uint64_t launches;    /* launches timed since the last reset */
    double total_ms;      /* sum of their CUDA-event durations */
    double alg_bytes;     /* algorithmic bytes those launches had to move (gate runs:
                             every touched column's x and z read and written once, the
                             sign column read and written, one 4-byte draw per noise op) */
} stab_kernel_stats;

/* Bracket every launch of the kernel kinds in `kind_mask` (bit k = kind k)
 * with CUDA events on its stream; 0 disables. */
int stab_profile(stab_ctx *ctx, uint32_t kind_mask);
/* Synchronize and return the accumulated statistics of one kernel kind. */
int stab_profile_read(stab_ctx *ctx, uint32_t kind, stab_kernel_stats *out, int reset);
/* Kernel launches issued by this context since the last reset. */
int stab_launch_count(stab_ctx *ctx, uint64_t *count, int reset);
/* Layered-engine work counters since the last reset (synchronizes); counted
 * only while per-launch profiling is on (stab_profile with a nonzero mask):
 * [0] random-measurement waves, [1] random measurements applied in waves,
 * [2] measurements found deterministic inside the random-measurement kernel,
 * [3] deterministic measurements resolved by the batched kernel,
 * [4] sum over deterministic measurements of |K| (stabilizer rows multiplied),
 * [5] sum over random measurements of |A| (rows that received a rowsum),
 * [6] cached pivots recomputed, [7] rowsum passes (one per wave), [8..15] SM clock cycles spent by
 * the random-measurement kernel in its per-wave phases (pending list with
 * the window pass [8], [9] unused, column and X-support rescans [10], [11]
 * unused, selection [12], work lists [13], rowsums with column updates and
 * row copies [14], the separate multi-pivot phase of serial waves [15]),
 * [16..18], [20], [21] sub-step cycles of the kernel's first warp,
 * [19] pivot-row X supports recomputed, [22] waves applied serially (a dense
 * pivot or an overflowed list), [23] waves with a dense pivot.
 * n <= 24 entries are written. */
int stab_engine_counters(stab_ctx *ctx, uint64_t *out, size_t n, int reset);

/* Read + write copy bandwidth of the context's device, for roofline
 * denominators: two buffers of bytes/2 each (allocated and freed inside the
 * call), one warm-up pass, then `passes` passes of a 16-byte-vector copy in
 * ONE launch, loads and stores through L2 only (ld/st .cg), timed with CUDA
 * events.  With bytes well below the L2 size every timed pass hits L2 (an L2
 * bandwidth figure); with bytes far above it every pass goes to HBM.
 * *gbs = 2 x (bytes/2) x passes / elapsed, in GB/s.  Synchronizes.  Errors:
 * STAB_ERR_ARG (bytes < 4096, passes = 0, gbs NULL), STAB_ERR_OOM. */
int stab_probe_copy(stab_ctx *ctx, uint64_t bytes, uint32_t passes, double *gbs);

#ifdef __cplusplus
}
#endif
#endif /* LIBSTAB_STAB_H_ */
