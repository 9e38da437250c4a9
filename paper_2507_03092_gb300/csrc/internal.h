// internal.h -- program format, device helpers and engine entry points shared
// by the translation units of libstab.so.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <map>
#include <memory>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/stab.h"

namespace stab {

// ---------------------------------------------------------------------------
// Compiled program
// ---------------------------------------------------------------------------
// A circuit is compiled into layers.  A gate layer holds items on pairwise
// disjoint qubits; each item is an optional Clifford gate followed by up to two
// noise ops on the same qubits.  A measurement layer holds M / R / RESET_ERROR
// ops on pairwise disjoint qubits.  Ops inside one layer commute exactly, so
// running a layer in parallel gives the same tableau, bit for bit, as running
// its ops one by one in circuit order.

enum LayerType : uint32_t { LT_GATE = 0, LT_MEAS = 1 };

// noise target of an item's noise op
enum : uint8_t { NT_A = 0, NT_B = 1, NT_AB = 2, NT_BA = 3 };
// measurement item flags
enum : uint32_t { MF_RESET = 1u, MF_RESET_ERR = 2u, MF_RESET_AFTER = 4u, MF_MPP = 8u };
// MF_MPP: a Pauli-product measurement; its factors are mfactors[nl, nl + np),
// each packed as qubit | code << 30 (code 1 X, 2 Y, 3 Z).
// MF_RESET_AFTER: an R that followed this M on the same qubit with no op on the
// qubit in between was folded in: that R is deterministic with this M's outcome,
// so it reduces to X after the measurement when the outcome is 1.

struct GItem {            // 32 bytes
    uint32_t a, b;        // qubits (b == a for one-qubit items)
    uint8_t gate;         // stab_kind of the gate, 0 = none
    uint8_t nn;           // noise ops attached (0..2)
    uint8_t nk[2];        // their kinds (STAB_DEP1 / STAB_DEP2 / STAB_PC1)
    uint8_t nt[2];        // their targets (NT_*)
    uint16_t pad;
    uint32_t nl[2];       // noise-draw ordinals
    uint32_t np[2];       // parameter rows
};
static_assert(sizeof(GItem) == 32, "GItem layout");

struct MItem {            // 24 bytes
    uint32_t q;
    uint32_t coin;        // coin ordinal (M / R); unused for RESET_ERR
    uint32_t rec;         // record ordinal, 0xffffffff if not recorded
    uint32_t flags;       // MF_*
    uint32_t nl;          // RESET_ERR: ordinal of its first noise draw; MPP: first factor
    uint32_t np;          // RESET_ERR: parameter row; MPP: number of factors
};
static_assert(sizeof(MItem) == 24, "MItem layout");

struct Layer {
    uint32_t type, first, count, has_cond;   // has_cond: R or RESET_ERR items present
    uint32_t ev_off, ev_cap;                 // gate layers: noise-event slots [ev_off, ev_off+ev_cap)
    uint32_t n_noisy;                        // items carrying noise
    uint32_t uniform;                        // gate layers: the gate kind every item has, else 0
};

// Packed gate item for the layered engine's slice kernel (noise handled by
// the event pre-pass): ab = a | b << 16 with a, b the operands' slots
// (gate_slot below), g = gate kind.
struct SItem {
    uint32_t ab, g;
};

// Shared-memory slot of column j in the slice kernel: j with its low four bits
// XORed with a hash of bits 4..9.  A slice holds 8 bytes per column, so 16
// consecutive slots fill the 32 banks once.  Within every aligned block of 16
// columns the map is a permutation, which keeps loops over consecutive
// columns free of bank conflicts.  The columns that one gate layer touches
// are often every other qubit; the hash spreads them over all 16 bank pairs,
// and the compiler orders each layer's items so that every aligned group of
// 16 items reads 16 distinct bank pairs as far as the layer allows.  Slots
// stay below n rounded up to a multiple of 16.  For columns j = i + k * 1024
// the XOR is the same for every k.
__host__ __device__ __forceinline__ uint32_t gate_slot(uint32_t j) {
    const uint32_t m = j >> 4;
    return j ^ ((m ^ (m >> 2)) & 15u);
}

struct Thr {              // floor(p_i * 2^32) for the three parameters of a row
    unsigned long long t[3];
};

struct DevProg {          // by-value descriptor handed to kernels
    uint32_t n, H, CW, n_layers;
    const Layer *layers;
    const GItem *gitems;
    const MItem *mitems;
    const Thr *thr;
    const SItem *sitems;      // packed copy of gitems (layered engine)
    const uint32_t *sab;      // their qubit pairs alone (a | b << 16), read by uniform layers
    const uint32_t *item_layer; // layer index of each gate item
    uint32_t record_words, coin_words, noise_words, max_meas;
    uint32_t max_gitems, n_gitems, n_mitems, ev_total;
    const uint32_t *mfactors;   // MPP factors (MF_MPP items)
    uint32_t n_mfactors, pad;
    uint8_t *layer_rand;        // [n_layers] set by k_meas_rand in a layer with a random op
};

struct Run {              // layered engine schedule entry
    uint32_t type;        // LT_GATE: layers [l0, l1); LT_MEAS: layer l0
    uint32_t l0, l1;
    double alg_bytes;     // LT_GATE, per tableau: distinct columns x,z read+written,
                          // sign column read+written, 4 bytes per noise draw
};

struct HostProg {
    uint64_t id = 0;
    uint32_t n = 0, H = 0, CW = 0;
    std::vector<Layer> layers;
    std::vector<GItem> gitems;
    std::vector<MItem> mitems;
    std::vector<Thr> thr;
    std::vector<SItem> sitems;
    std::vector<uint32_t> sab;
    std::vector<uint32_t> item_layer;
    std::vector<Run> runs;
    std::vector<uint32_t> mfactors;
    // The layered engine runs a Pauli-product measurement as the Clifford
    // conjugation U^dag M_Z U of one qubit; `lay` is the program compiled
    // from that rewritten op list (null when the circuit has no MPP).
    std::unique_ptr<HostProg> lay;
    // Layered-engine launch sequence replayed as a CUDA graph.  The graph is
    // valid for the kernel arguments and entry state in `gkey`; a different
    // key recaptures it and updates the executable graph in place once its
    // last launch has finished (event `gdone`); a different wave-kernel cluster
    // size instantiates it anew instead (a launch attribute, not updated).
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t gdone = nullptr;
    std::vector<unsigned char> gkey;
    unsigned long long glaunches = 0;   // kernel launches in the graph
    bool grm_after = false;             // batch's row-packed copy valid after the run
    uint32_t gcl = 0;                   // wave-kernel cluster size the executable graph was built with
    // Measurement layers that never have a random outcome.  Whether a Z
    // measurement is random depends only on the stabilizer group up to signs,
    // which Pauli noise, measurement outcomes and the X of resets leave alone:
    // from |0...0>, it is fixed by the circuit unless the circuit holds
    // RESET_ERROR (whose reset happens or not by a noise draw).  k_meas_rand
    // marks each layer that has a random op (dev.layer_rand); after a run
    // from |0...0> without device errors the host reads the marks once, and
    // later such runs leave out the random-measurement launches of unmarked
    // layers (and the stabilizer half of their measured columns, see
    // DET_SKIPPED; a random op there fails k_meas_det's product check).
    bool rand_learn = false;            // the circuit allows it (no RESET_ERROR)
    int rand_state = 0;                 // 0 unknown, 1 read-back queued, 2 known
    cudaEvent_t rand_ev = nullptr;
    uint8_t *rand_host = nullptr;       // pinned: [n_layers] marks, then the device error flag (int)
    std::vector<uint8_t> rand_skip;     // per layer: leave out k_destab_to_rm, k_meas_rand, k_meas_late
    stab_circuit_info info{};
    uint64_t cost = 0;          // rough work estimate (for scheduling)
    void *dmem = nullptr;       // device copy of the arrays
    DevProg dev{};
};

// Compile ops -> HostProg (host only).  Returns STAB_OK or an error code and
// writes a message to *err.
int compile_program(uint32_t n, const stab_op *ops, size_t n_ops, const double *params,
                    size_t n_params, HostProg &out, std::string *err);
// The program the layered engine runs (the conjugated form if there is one).
inline const HostProg &layered_prog(const HostProg &p) { return p.lay ? *p.lay : p; }

// ---------------------------------------------------------------------------
// Streams
// ---------------------------------------------------------------------------
struct DevStreams {
    uint32_t mode, pad;
    unsigned long long seed, shot_offset;
    const unsigned long long *coins;
    unsigned long long coin_stride;
    const uint32_t *noise;
    unsigned long long noise_stride;
};

// ---------------------------------------------------------------------------
// Layered engine storage (one batch of tableaux with the same n)
// ---------------------------------------------------------------------------
// Column-packed copy ("QM"): for tableau t, plane x then plane z, each
// [CW][n] 32-bit words; word w of column j holds rows 32w..32w+31 of column j.
// Row-packed copy ("RM"): [64H rows][2H words] (x words then z words).
// Row slots: destabilizer i -> slot i, stabilizer i -> slot 32H + i.
// Sign bits r: [CW] words over row slots.  dirty[w] = 1 when the row-packed
// copy of rows 32w..32w+31 is newer than the column-packed one.
struct Batch {
    uint32_t n = 0, H = 0, CW = 0, count = 0;
    uint32_t *qm = nullptr;  size_t qm_stride = 0;   // words per tableau
    uint32_t *rm = nullptr;  size_t rm_stride = 0;
    uint32_t *r = nullptr;
    uint8_t *dirty = nullptr;
    uint32_t *tflags = nullptr;   // per tableau: bit 0 destabilizer half of RM current,
                                  // bit 1 the current measurement layer has random ops
    bool rm_valid = false;
    void *mem = nullptr;
    size_t bytes = 0;             // bytes the current layout uses
    size_t cap = 0;               // bytes allocated (a smaller layout reuses them)
};

struct MeasScratch {
    uint32_t *cols = nullptr;     // [count][max_meas][CW]
    uint8_t *stat = nullptr;      // [count][max_meas]
    uint8_t *out = nullptr;       // [count][max_meas]
    uint16_t *mxs = nullptr;      // [count][max_meas][XSCAP] layer items j with X on q_j in the op's pivot row
    uint8_t *mxn = nullptr;       // [count][max_meas] entries of mxs (XS_OVER: more than XSCAP, XS_UNKNOWN: not computed)
    uint32_t *mxver = nullptr;    // [count][max_meas] version of the pivot row when mxs was computed
    uint32_t *rowver = nullptr;   // [count][32H] stabilizer-row versions (bumped whenever a row changes)
    uint16_t *qmap = nullptr;     // [count][n] qubit -> item of the current layer (0xffff: none)
    uint32_t *mpiv = nullptr;     // [count][max_meas] cached pivot (slot - 32H) or ~0
    uint32_t *mbsz = nullptr;     // [count][max_meas] cached |x-column support|
    uint8_t *mstale = nullptr;    // [count][max_meas] cache invalid
    uint16_t *msup = nullptr;     // [count][max_meas][SUPCAP] column support rows (if small)
    uint16_t *pwl = nullptr;      // [count][WCAP_MAX][PWCAP] nonzero words of the wave's pivot rows
    uint32_t *flips = nullptr;    // [count][2*max_meas] qubit | Pauli<<30 to apply after the layer
    uint32_t *flip_cnt = nullptr; // [count][n_layers]
    uint32_t *ev = nullptr;       // [count][ev_total] noise events
    uint32_t *ev_cnt = nullptr;   // [count][n_layers] noise-event counts
    struct CallArgs *call = nullptr;   // per-call inputs of the layered engine (device)
    size_t cap_words = 0, cap_items = 0;
};

// Inputs that change from call to call (streams, record buffer): kept in
// device memory, written before each run, so a captured launch sequence can be
// replayed unchanged.
struct CallArgs {
    DevStreams st;
    unsigned long long *record;
    unsigned long long rec_stride;
};

struct LaunchCfg {
    int sm_count = 0;
    size_t smem_optin = 0;
    uint32_t rand_cluster = 1;    // CTAs per tableau of the random-measurement kernel (set per run)
};

// Capacities of the random-measurement wave kernel's shared-memory lists.
// Overflowing a list is handled by slower fallback loops; tests shrink the
// capacities (STAB_WAVE_CAPS="pcap,wcap,paircap,jcap,budget[,window[,wave_limit]]")
// to exercise them.
struct WaveCaps {
    // Maxima size k_meas_rand's shared memory, which shares each SM's 256 KB
    // with its L1 cache; larger lists only fall back to slower loops when
    // they overflow.  The window (pending measurements examined per wave,
    // at most WINDOW_MAX) may hold more selectable measurements than a wave
    // takes (WCAP_MAX): those beyond it stay pending for the next wave.
    static constexpr uint32_t PCAP_MAX = 4096, WCAP_MAX = 512, PAIRCAP_MAX = 2048, JCAP_MAX = 2048,
                              WINDOW_MAX = 1024;
    uint32_t pcap = PCAP_MAX;          // pending measurements considered per wave
    uint32_t wcap = WCAP_MAX;          // measurements applied per wave
    uint32_t paircap = PAIRCAP_MAX;    // (row, pivot) rowsum pairs listed per wave
    uint32_t jcap = JCAP_MAX;          // measured-column updates listed per wave
    uint32_t mark_budget = 0;          // unused (kept so that the test variable keeps its fields)
    uint32_t window = WINDOW_MAX;      // pending measurements examined per wave
    // Waves allowed per measurement layer before the kernel gives up with a
    // bounds error (the loop's own bound, 2 x ops + 3, applies as well);
    // lowered only by tests, to see the guard fire and the context survive.
    uint32_t wave_limit = 0xffffffffu;
};
constexpr uint32_t SUPCAP = 64;        // rows kept in a measured column's support list (two per lane of a warp)
constexpr uint32_t PWCAP = 64;         // nonzero words kept per pivot row
constexpr uint32_t XSCAP = 32;         // layer items kept per pivot-row X support
constexpr uint8_t XS_OVER = 0xff, XS_UNKNOWN = 0xfe;
void set_wave_caps(const WaveCaps &c);

// Launch accounting and optional per-kernel CUDA-event timing.
struct KernelProf {
    uint32_t mask = 0;
    unsigned long long launches = 0;          // every launch, timed or not
    struct Rec { uint32_t kind; cudaEvent_t e0, e1; double bytes; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    unsigned long long n[STAB_N_KERNEL_KINDS] = {};
    double ms[STAB_N_KERNEL_KINDS] = {};
    double bytes[STAB_N_KERNEL_KINDS] = {};
    std::mutex mu;
    cudaEvent_t take();
    void begin(uint32_t kind, cudaStream_t s, Rec &r);
    void end(Rec &r, cudaStream_t s, double bytes);
    int collect();                            // synchronizes pending events
};

// Raise a kernel's dynamic shared-memory limit to `bytes` once per (slot,
// current device): the attribute is per device, and contexts on several
// devices or host threads launch the same kernels.  Allocates nothing.
void smem_attr_once(int slot, const void *func, int bytes);

size_t batch_bytes(uint32_t n, uint32_t count);
int batch_alloc(Batch &b, uint32_t n, uint32_t count, std::string *err);
void batch_free(Batch &b);

// Layered engine (layered.cu)
cudaError_t layered_init(Batch &b, cudaStream_t s, KernelProf *kp);
// A capturable stream joined to the caller's stream by two events: the
// layered engine captures its launch sequence there and replays it as a graph.
struct GraphSlot {
    cudaStream_t gs = nullptr;
    cudaEvent_t in = nullptr, out = nullptr;
};
int graph_slot_init(GraphSlot &g);
void graph_slot_free(GraphSlot &g);
void prog_graphs_free(HostProg &p);
// gsl: replay as a CUDA graph through this slot when per-launch profiling is
// off (nullptr: plain launches on s)
cudaError_t layered_run(const HostProg &p, Batch &b, MeasScratch &ms, const DevStreams &st,
                        unsigned long long *record, size_t rec_stride, int *d_err,
                        const LaunchCfg &lc, cudaStream_t s, KernelProf *kp,
                        unsigned long long *d_stats, GraphSlot *gsl = nullptr, bool fresh = false);
cudaError_t layered_sync_qm(Batch &b, cudaStream_t s);
cudaError_t layered_commute(Batch &b, uint32_t index, const unsigned long long *px, const unsigned long long *pz,
                            size_t m, unsigned long long *out, cudaStream_t s, KernelProf *kp);
size_t layered_gate_smem(uint32_t n);
int layered_supported(uint32_t n, const LaunchCfg &lc);

// Resident engine (resident.cu)
struct ResJob {               // one shot
    const DevProg *prog;      // device pointer
    DevStreams st;            // streams of its group (shot index below)
    unsigned long long *record;
    unsigned long long rec_stride;
    uint32_t shot;            // shot index within its group
    uint32_t pad;
};
size_t resident_smem_per_tableau(uint32_t n);
int resident_supported(uint32_t n, const LaunchCfg &lc);
int resident_shape_ok(uint32_t max_n, const stab_tune &tune, const LaunchCfg &lc);
cudaError_t resident_run(const ResJob *d_jobs, uint32_t n_jobs, uint32_t max_n,
                         const stab_tune &tune, unsigned int *d_counter, int *d_err,
                         const LaunchCfg &lc, cudaStream_t s, KernelProf *kp);

// device counters (unsigned long long) kept next to the error flag
// DC_PHASE0 + k: SM cycles of k_meas_rand's per-wave phase k (0 pending list,
// 1 cached-state pass, 2 column rescans, 3 X-support rescans, 4 selection,
// 5 work lists, 6 single-pivot rows + column updates + row copies,
// 7 multi-pivot rows)
enum : int { DC_WAVES = 0, DC_WAVE_OPS = 1, DC_DET_NOW = 2, DC_DET = 3, DC_SUM_K = 4, DC_SUM_A = 5,
             DC_PIV_RECOMP = 6, DC_ROWSUM_PASSES = 7, DC_PHASE0 = 8, DC_N_PHASES = 11,
             DC_XS_RECOMP = 19, DC_N = 24,
             // SM cycles of warp 0's sub-steps: work lists (row scans, pair lists),
             // multi-pivot rows (chain walk and keys, sort, scan rows)
             DC_W0_LIST_SCAN = 16, DC_W0_LIST_PAIRS = 17, DC_W0_MULTI_WALK = 18, DC_W0_MULTI_SORT = 20,
             DC_W0_MULTI_ROWS = 21, DC_SERIAL_WAVES = 22, DC_DENSE_WAVES = 23 };

// device error flag values
enum : int { DERR_NONE = 0, DERR_ODD_PHASE = 1, DERR_BAD_PRODUCT = 2, DERR_TIMEOUT = 3,
             DERR_BOUNDS = 4 };

}  // namespace stab
