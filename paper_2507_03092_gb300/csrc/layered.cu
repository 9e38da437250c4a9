// layered.cu -- the layered engine: a batch of tableaux in device memory,
// one launch per run of gate layers and a few per measurement layer.
//
// Layout (see internal.h): a column-packed copy (QM, 32 rows of one column
// per word) serves the Clifford layers, whose updates are column-wise
// (Sec. 2.4: "Hadamard, phase and CNOT operations occur on every row of the
// tableau, at the column that the gate targets"); a row-packed copy (RM)
// serves measurement, whose rowsum (Appendix B) works on whole rows.
//
//  * k_gate_run: one CTA per (32-row slice, tableau).  The slice -- word w of
//    every column -- is staged in shared memory, the whole run of gate layers
//    is applied to it (gates are row-independent, Sec. 3.1.1, so no other CTA
//    is involved), and the slice is written back column-packed and, when a
//    measurement layer follows, row-packed (32x32 warp transposes).
//  * k_meas_det: one warp per measurement.  Pivot search (Sec. 3.1.2) on the
//    measured column; for deterministic outcomes the sign of the product of
//    the stabilizers selected by the destabilizer column (Sec. 2.4, rowsum into
//    a scratch row) is computed in one pass with the ordered-product closed
//    form instead of Alg. 2's per-row grid synchronisation.  Deterministic
//    outcomes do not depend on the other Z measurements of the layer.
//  * k_meas_rand: one CTA per tableau runs the layer's random measurements
//    (pivot, rowsum of the pivot into every anticommuting row with the mod-4
//    phase, destabilizer copy, +-Z_a install; Sec. 2.4) in waves.  Two random
//    measurements s, t commute as tableau operations when neither pivot row
//    has an X or Y on the other's qubit: each leaves the other's pivot and
//    measured column unchanged (up to the overwritten destabilizer partner),
//    and a row both multiply receives the product of two commuting pivots,
//    whose sign does not depend on the order.  A pending measurement joins the
//    current wave when it commutes in this sense with every earlier pending
//    one, so applying the wave at once gives the tableau circuit order gives,
//    bit for bit.  The measured columns of the remaining ops are kept current
//    from the pivot rows.
//  * k_noise_events: noise draws are evaluated once per shot before the gate
//    runs; the few Pauli errors that fire are listed per layer and applied by
//    the slice kernels after the layer's gates.
//  * k_cond: the X of resets whose outcome was 1 (and the Z of RESET_ERROR)
//    as sign flips r ^= z_a (x_a); these Paulis commute with the layer's other
//    measurements, so they are applied after it -- by the next gate run as it
//    loads each slice when one follows, else by this kernel.
#include "device_common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

namespace cg = cooperative_groups;

namespace stab {

enum : uint8_t { MS_DONE = 0, MS_RANDOM = 1, MS_SKIP = 2, MS_WAVE = 3, MS_DETLATE = 4 };
// layer | DET_SKIPPED (k_gather_cols, k_meas_det): the circuit has shown that
// the layer has no random op, so its random-measurement kernels are left out
// and only the destabilizer half of each measured column is gathered and
// scanned: its set rows name the stabilizers whose product is +-Z_a.  Were
// an op random after all, that product would not be +-Z_a (Z_a would not be
// in the stabilizer group), which the product check reports.
constexpr uint32_t DET_SKIPPED = 0x80000000u;
// MS_DETLATE: an op that was random when the layer started but became
// deterministic after earlier random ops of the layer.  Its outcome does not
// change under the layer's remaining Z measurements, so k_meas_late resolves
// all of them after k_meas_rand, one warp each across the whole GPU; until then
// their measured columns are kept current like those of pending random ops.
// tflags: the row-packed copy's destabilizer half (rows of slices w < H) is
// only needed by random measurements; gate runs write the stabilizer half and
// k_destab_to_rm fills the other half when a layer turns out to have random ops.
enum : uint32_t { TF_DESTAB_FRESH = 1u, TF_RAND_LAYER = 2u };


struct LArgs {
    DevProg P;
    uint32_t *qm;
    unsigned long long qm_stride;
    uint32_t *rm;
    unsigned long long rm_stride;
    uint32_t RS, Hr;                 // row stride (words) and z offset in a row
    uint32_t *r;
    uint8_t *dirty;
    uint32_t *tflags;                // TF_* per tableau
    uint32_t *cols;
    unsigned long long cols_stride;  // words per tableau
    uint8_t *mstat, *mout;
    unsigned long long m_stride;     // items per tableau
    uint16_t *mxs;                   // [B][max_meas][XSCAP] pivot-row X support over the layer's items
    uint8_t *mxn;                    // [B][max_meas] its length, XS_OVER or XS_UNKNOWN
    uint32_t *mxver;                 // [B][max_meas] pivot-row version it was computed at
    uint32_t *rowver;                // [B][32H] stabilizer-row versions
    uint16_t *qmap;                  // [B][n]
    uint32_t *ev, *ev_cnt;           // [B][ev_total], [B][n_layers]
    uint32_t *mpiv, *mbsz;           // [B][max_meas] cached pivot / column size
    uint8_t *mstale;                 // [B][max_meas]
    uint16_t *msup;                  // [B][max_meas][SUPCAP]
    uint16_t *pwl;                   // [B][WCAP_MAX][PWCAP]
    uint32_t *flips, *flip_cnt;      // [B][2*max_meas], [B][n_layers]
    unsigned long long *stats;       // DC_* counters (may be null)
    WaveCaps caps;                   // k_meas_rand list capacities (<= compile-time maxima)
    const CallArgs *call;            // streams and record of this call (device)
    int *err;
    uint32_t B;
};

static inline uint32_t round4(uint32_t v) { return (v + 3u) & ~3u; }
extern WaveCaps g_caps;

__device__ __forceinline__ uint32_t rbit(const uint32_t *r, uint32_t s) {
    return (r[s >> 5] >> (s & 31)) & 1u;
}

// ---------------------------------------------------------------- init
__global__ void k_init(LArgs a) {
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW, RS = a.RS, Hr = a.Hr;
    const unsigned long long qm_per = (unsigned long long)CW * n;
    const unsigned long long rm_rows = 64ull * H;
    const unsigned long long gsz = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long start = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t t = 0; t < a.B; t++) {
        uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + qm_per;
        for (unsigned long long e = start; e < qm_per; e += gsz) {
            uint32_t w = (uint32_t)(e / n), j = (uint32_t)(e % n);
            uint32_t bit = 1u << (j & 31);
            qx[e] = (w == (j >> 5)) ? bit : 0u;
            qz[e] = (w == H + (j >> 5)) ? bit : 0u;
        }
        uint32_t *rm = a.rm + t * a.rm_stride;
        for (unsigned long long e = start; e < rm_rows * RS; e += gsz) {
            uint32_t s = (uint32_t)(e / RS), c = (uint32_t)(e % RS);
            uint32_t v = 0;
            if (s < n) {
                if (c == (s >> 5)) v = 1u << (s & 31);
            } else if (s >= 32 * H && s - 32 * H < n) {
                uint32_t i = s - 32 * H;
                if (c == Hr + (i >> 5)) v = 1u << (i & 31);
            }
            rm[e] = v;
        }
        for (unsigned long long e = start; e < CW; e += gsz) {
            a.r[(unsigned long long)t * CW + e] = 0u;
            a.dirty[(unsigned long long)t * CW + e] = 0;
        }
        if (start == 0) a.tflags[t] = TF_DESTAB_FRESH;
    }
}

// ---------------------------------------------------------------- transposes
// Write rows 32w..32w+31 of the row-packed copy from column words given by
// `col(j)` (word w of column j, 0 for j >= n).  One warp handles 4 consecutive
// column blocks so every lane stores 16 contiguous bytes of its row.
template <typename ColX, typename ColZ>
__device__ __forceinline__ void slice_store_rm(uint32_t *rm, uint32_t RS, uint32_t Hr, uint32_t H,
                                               uint32_t w, ColX colx, ColZ colz) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t row = 32 * w + lane;
    for (uint32_t c0 = 4 * warp; c0 < H; c0 += 4 * nw) {
        uint4 vx, vz;
        vx.x = warp_transpose32(colx(32 * (c0 + 0) + lane));
        vx.y = warp_transpose32(colx(32 * (c0 + 1) + lane));
        vx.z = warp_transpose32(colx(32 * (c0 + 2) + lane));
        vx.w = warp_transpose32(colx(32 * (c0 + 3) + lane));
        vz.x = warp_transpose32(colz(32 * (c0 + 0) + lane));
        vz.y = warp_transpose32(colz(32 * (c0 + 1) + lane));
        vz.z = warp_transpose32(colz(32 * (c0 + 2) + lane));
        vz.w = warp_transpose32(colz(32 * (c0 + 3) + lane));
        *reinterpret_cast<uint4 *>(rm + (size_t)row * RS + c0) = vx;
        *reinterpret_cast<uint4 *>(rm + (size_t)row * RS + Hr + c0) = vz;
    }
}

// Read rows 32w..32w+31 of the row-packed copy and hand column words to
// `put(j, xword, zword)` for j < n.
template <typename Put>
__device__ __forceinline__ void slice_load_rm(const uint32_t *rm, uint32_t RS, uint32_t Hr, uint32_t H,
                                              uint32_t n, uint32_t w, Put put) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t row = 32 * w + lane;
    for (uint32_t c0 = 4 * warp; c0 < H; c0 += 4 * nw) {
        uint4 vx = *reinterpret_cast<const uint4 *>(rm + (size_t)row * RS + c0);
        uint4 vz = *reinterpret_cast<const uint4 *>(rm + (size_t)row * RS + Hr + c0);
        uint32_t xs[4] = {vx.x, vx.y, vx.z, vx.w}, zs[4] = {vz.x, vz.y, vz.z, vz.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            uint32_t cx = warp_transpose32(xs[k]);
            uint32_t cz = warp_transpose32(zs[k]);
            uint32_t j = 32 * (c0 + k) + lane;
            if (j < n) put(j, cx, cz);
        }
    }
}

// word w of column q from the row-packed copy (x plane, or z plane if zp)
__device__ __forceinline__ uint32_t rm_col_word(const uint32_t *rm, uint32_t RS, uint32_t Hr,
                                                uint32_t w, uint32_t q, bool zp) {
    uint32_t v = 0;
    const uint32_t off = (zp ? Hr : 0u) + (q >> 5), sh = q & 31;
    for (uint32_t k = 0; k < 32; k++)
        v |= ((rm[(size_t)(32 * w + k) * RS + off] >> sh) & 1u) << k;
    return v;
}

// ---------------------------------------------------------------- gate runs
struct GRun {
    uint32_t l0, l1, want_rm;
    int32_t cond_layer;     // measurement layer whose reset/RESET_ERROR flips act first, or -1
};

// Combined Pauli (2-bit x|z<<1 form) of an item's noise ops on its two qubits.
__device__ __forceinline__ void item_noise(const GItem &g, const DevStreams &st, uint32_t shot,
                                           const Thr *thr, uint32_t &Pa, uint32_t &Pb) {
    // Pauli code (1 X, 2 Y, 3 Z) -> x | z << 1 is code ^ (code >> 1)
    Pa = 0; Pb = 0;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        if (k >= g.nn) break;
        const uint32_t u = noise_word(st, shot, k ? g.nl[1] : g.nl[0]);
        int pa, pb;
        noise_paulis(k ? g.nk[1] : g.nk[0], u, thr[k ? g.np[1] : g.np[0]], pa, pb);
        if (!(pa | pb)) continue;
        const uint32_t xa = (uint32_t)(pa ^ (pa >> 1)), xb = (uint32_t)(pb ^ (pb >> 1));
        switch (k ? g.nt[1] : g.nt[0]) {
        case NT_A: Pa ^= xa; break;
        case NT_B: Pb ^= xa; break;
        case NT_AB: Pa ^= xa; Pb ^= xb; break;
        default: Pb ^= xa; Pa ^= xb; break;
        }
    }
}

__device__ __forceinline__ uint32_t xz_flip(uint32_t P, uint32_t x, uint32_t z) {
    return ((P & 1u) ? z : 0u) ^ ((P & 2u) ? x : 0u);
}

// One thread per gate item (x all tableaux): evaluate its noise draws and list
// the Pauli errors that fire under the item's layer.  A layer whose events
// overflow its slots keeps counting; the slice kernel then re-evaluates it.
__global__ void k_noise_events(LArgs a) {
    const unsigned long long total = (unsigned long long)a.P.n_gitems * a.B;
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(e / a.P.n_gitems), i = (uint32_t)(e % a.P.n_gitems);
        const GItem g = a.P.gitems[i];
        if (!g.nn) continue;
        uint32_t Pa, Pb;
        item_noise(g, a.call->st, t, a.P.thr, Pa, Pb);
        if (!(Pa | Pb)) continue;
        const uint32_t l = a.P.item_layer[i];
        const Layer L = a.P.layers[l];
        uint32_t *cnt = a.ev_cnt + (size_t)t * a.P.n_layers + l;
        uint32_t *ev = a.ev + (size_t)t * a.P.ev_total + L.ev_off;
        if (Pa) {
            const uint32_t k = atomicAdd(cnt, 1u);
            if (k < L.ev_cap) ev[k] = g.a | (Pa << 30);
        }
        if (Pb) {
            const uint32_t k = atomicAdd(cnt, 1u);
            if (k < L.ev_cap) ev[k] = g.b | (Pb << 30);
        }
    }
}

// The gate items of one layer on a slice held in shared memory (items in
// groups of 4 per thread, all four loaded before any is used).  KIND != 0:
// every item of the layer is that gate (no per-item dispatch).
template <uint32_t KIND>
__device__ __forceinline__ void gate_items(const uint2 *__restrict__ it, uint32_t count, uint2 *sxz,
                                           uint32_t &racc) {
    for (uint32_t i0 = threadIdx.x; i0 < count; i0 += 4 * blockDim.x) {
        uint2 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t i = i0 + k * blockDim.x;
            v[k] = i < count ? __ldg(it + i) : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t ga = v[k].x & 0xffffu, gb = v[k].x >> 16, gk = v[k].y;
            if (!gk) continue;
            const uint2 va = sxz[ga];
            uint32_t xa = va.x, za = va.y, xb = 0, zb = 0;
            const bool two = gb != ga;
            if (two) {
                const uint2 vb = sxz[gb];
                xb = vb.x;
                zb = vb.y;
            }
            racc ^= apply_gate(gk, xa, za, xb, zb);
            sxz[ga] = make_uint2(xa, za);
            if (two) sxz[gb] = make_uint2(xb, zb);
        }
    }
}

// A uniform layer (every item the same gate KIND): 4-byte qubit pairs, eight
// per thread loaded before any is used, so a layer of up to 8 x blockDim items
// costs one round trip for its items.
template <uint32_t KIND>
__device__ __forceinline__ void gate_items_u(const uint32_t *__restrict__ ab, uint32_t count, uint2 *sxz,
                                             uint32_t &racc) {
    for (uint32_t i0 = threadIdx.x; i0 < count; i0 += 8 * blockDim.x) {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t i = i0 + k * blockDim.x;
            v[k] = i < count ? __ldg(ab + i) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (i0 + k * blockDim.x >= count) break;
            const uint32_t ga = v[k] & 0xffffu, gb = v[k] >> 16;
            if (KIND == STAB_H || KIND == STAB_S) {
                const uint2 va = sxz[ga];
                uint32_t xa = va.x, za = va.y, xb = 0, zb = 0;
                racc ^= apply_gate(KIND, xa, za, xb, zb);
                sxz[ga] = make_uint2(xa, za);
            } else {
                const uint2 va = sxz[ga], vb = sxz[gb];
                uint32_t xa = va.x, za = va.y, xb = vb.x, zb = vb.y;
                racc ^= apply_gate(KIND, xa, za, xb, zb);
                sxz[ga] = make_uint2(xa, za);
                sxz[gb] = make_uint2(xb, zb);
            }
        }
    }
}

// A layer whose noise events overflowed their slots: every draw of the layer
// evaluated again (kept out of line: the common path needs none of this).
__device__ __noinline__ uint32_t layer_noise_all(const GItem *items, uint32_t count, const Thr *thr,
                                                 const CallArgs *call, uint32_t t, const uint2 *sxz) {
    uint32_t racc = 0;
    for (uint32_t k = threadIdx.x; k < count; k += blockDim.x) {
        const GItem gi = items[k];
        if (!gi.nn) continue;
        uint32_t Pa, Pb;
        item_noise(gi, call->st, t, thr, Pa, Pb);
        const uint2 va = sxz[gate_slot(gi.a)], vb = sxz[gate_slot(gi.b)];
        racc ^= xz_flip(Pa, va.x, va.y) ^ xz_flip(Pb, vb.x, vb.y);
    }
    return racc;
}

constexpr uint32_t RUN_STAGE = 16;       // layers of a run whose descriptors are staged
// FIXED: blockDim.x is 1024, so the slot of every column a thread visits in
// its strided loops is the column XOR one per-thread constant.
template <bool FIXED>
__global__ void __launch_bounds__(1024, 2) k_gate_run(LArgs a, GRun g) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t sred[32];
    __shared__ Layer s_layer[RUN_STAGE];
    __shared__ uint32_t s_evc[RUN_STAGE];
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW;
    // stabilizer-half slices (which also write the row-packed copy) first, so
    // that the last, partial wave of CTAs holds the lighter ones (2.4 % per
    // d = 71 step on GB300: 632 slices fill 2.08 waves of 2 CTAs per SM)
    const uint32_t w = (blockIdx.x + H) % CW, t = blockIdx.y;
    // the run's first layers (descriptors and noise-event counts), staged
    // while the slice loads
    if (threadIdx.x < min(RUN_STAGE, g.l1 - g.l0)) {
        const uint32_t l = g.l0 + threadIdx.x;
        s_layer[threadIdx.x] = a.P.layers[l];
        s_evc[threadIdx.x] = a.ev_cnt ? a.ev_cnt[(size_t)t * a.P.n_layers + l] : 0u;
    }
    // the slice: word w of column j's x and z planes side by side in slot
    // gate_slot(j) (one 8-byte shared-memory access per column and gate
    // operand; the items carry their operands' slots)
    uint2 *sxz = reinterpret_cast<uint2 *>(smem);
    const uint32_t tx = gate_slot(threadIdx.x) ^ threadIdx.x;
    // slot of column j in the loops over j = threadIdx.x + k * blockDim.x
    auto cslot = [&](uint32_t j) { return FIXED ? (j ^ tx) : gate_slot(j); };
    uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + (size_t)CW * n;
    uint32_t *rm = a.rm + t * a.rm_stride;
    uint8_t *dirty = a.dirty + (size_t)t * CW;
    const bool dty = dirty[w] != 0;
    if (!dty) {
        // four words of each plane loaded per thread before any is stored, so
        // that each thread keeps 32 bytes in flight (one pair at a time keeps
        // too few bytes in flight per SM to cover the DRAM latency)
        const uint32_t *__restrict__ gx = qx + (size_t)w * n;
        const uint32_t *__restrict__ gz = qz + (size_t)w * n;
        const uint32_t bd = blockDim.x;
        for (uint32_t j0 = threadIdx.x; j0 < n; j0 += 4 * bd) {
            uint32_t vx[4], vz[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t j = j0 + k * bd;
                vx[k] = j < n ? gx[j] : 0u;
                vz[k] = j < n ? gz[j] : 0u;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t j = j0 + k * bd;
                if (j < n) sxz[cslot(j)] = make_uint2(vx[k], vz[k]);
            }
        }
    } else {
        slice_load_rm(rm, a.RS, a.Hr, H, n, w,
                      [&](uint32_t j, uint32_t x, uint32_t z) { sxz[gate_slot(j)] = make_uint2(x, z); });
    }
    __syncthreads();
    uint32_t racc = 0;
    if (g.cond_layer >= 0) {
        // X after resets with outcome 1 and RESET_ERROR's Z from the preceding
        // measurement layer: sign flips on the rows anticommuting with them,
        // applied before this run's first gate
        const uint32_t cnt = a.flip_cnt[(size_t)t * a.P.n_layers + (uint32_t)g.cond_layer];
        const uint32_t *fl = a.flips + t * 2 * a.m_stride;
        for (uint32_t e = threadIdx.x; e < cnt; e += blockDim.x) {
            const uint32_t f = fl[e];
            const uint2 v = sxz[gate_slot(f & 0x3fffffffu)];
            racc ^= (f >> 30) == 1u ? v.y : v.x;
        }
        __syncthreads();          // every flip has read its pre-gate word
    }
    for (uint32_t l = g.l0; l < g.l1; l++) {
        const bool staged = l - g.l0 < RUN_STAGE;
        const Layer L = staged ? s_layer[l - g.l0] : a.P.layers[l];
        // the layer's Pauli errors (a few dozen at most per layer, normally):
        // counts staged above, one event per thread loaded before the gates run
        uint32_t ecnt = 0, my_ev = 0;
        if (L.n_noisy) {
            ecnt = staged ? s_evc[l - g.l0] : a.ev_cnt[(size_t)t * a.P.n_layers + l];
            if (ecnt <= L.ev_cap && threadIdx.x < ecnt)
                my_ev = a.ev[(size_t)t * a.P.ev_total + L.ev_off + threadIdx.x];
        }
        // gates: packed items through the read-only path
        const uint2 *__restrict__ it = reinterpret_cast<const uint2 *>(a.P.sitems + L.first);
        // items in groups of 4 per thread, all four loaded before any is used;
        // layers made of one gate kind (every layer of a surface-code round)
        // run a loop specialised to it
        const uint32_t *__restrict__ iab = a.P.sab + L.first;
        switch (L.uniform) {
        case STAB_H: gate_items_u<STAB_H>(iab, L.count, sxz, racc); break;
        case STAB_CX: gate_items_u<STAB_CX>(iab, L.count, sxz, racc); break;
        case STAB_CZ: gate_items_u<STAB_CZ>(iab, L.count, sxz, racc); break;
        case STAB_S: gate_items_u<STAB_S>(iab, L.count, sxz, racc); break;
        default: gate_items<0>(it, L.count, sxz, racc); break;
        }
        __syncthreads();
        if (L.n_noisy) {
            // the layer's Pauli errors act after its gates
            const uint32_t cnt = ecnt;
            if (cnt <= L.ev_cap) {
                if (threadIdx.x < cnt) {
                    const uint2 v = sxz[gate_slot(my_ev & 0x3fffffffu)];
                    racc ^= xz_flip(my_ev >> 30, v.x, v.y);
                }
                const uint32_t *ev = a.ev + (size_t)t * a.P.ev_total + L.ev_off;
                for (uint32_t e = threadIdx.x + blockDim.x; e < cnt; e += blockDim.x) {
                    const uint32_t v = ev[e];
                    const uint2 c = sxz[gate_slot(v & 0x3fffffffu)];
                    racc ^= xz_flip(v >> 30, c.x, c.y);
                }
            } else {
                racc ^= layer_noise_all(a.P.gitems + L.first, L.count, a.P.thr, a.call, t, sxz);
            }
            __syncthreads();
        }
    }
    // sign flips: XOR-reduce over the CTA, one plain update per slice
    racc = __reduce_xor_sync(FULL_MASK, racc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sred[warp] = racc;
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
        const uint2 v = sxz[cslot(j)];
        qx[(size_t)w * n + j] = v.x;
        qz[(size_t)w * n + j] = v.y;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < nw ? sred[lane] : 0u;
        v = __reduce_xor_sync(FULL_MASK, v);
        if (lane == 0) {
            a.r[(size_t)t * CW + w] ^= v;
            dirty[w] = 0;
        }
    }
    if (w == 0 && threadIdx.x == 0) a.tflags[t] &= ~TF_DESTAB_FRESH;
    if (g.want_rm && w >= H) {        // stabilizer half only (see TF_DESTAB_FRESH)
        slice_store_rm(rm, a.RS, a.Hr, H, w,
                       [&](uint32_t j) { return j < n ? sxz[gate_slot(j)].x : 0u; },
                       [&](uint32_t j) { return j < n ? sxz[gate_slot(j)].y : 0u; });
    }
}

// Destabilizer half of the row-packed copy, for tableaux whose current
// measurement layer has random ops and whose copy is stale.  The column-packed
// copy is current then: it is only left behind by random measurements, which
// first make the destabilizer half current.
// (a fixed grid striding over the (tableau, slice) pairs: most tableaux need
// nothing here)
__global__ void k_destab_to_rm(LArgs a) {
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW;
    for (unsigned long long pidx = blockIdx.x; pidx < (unsigned long long)H * a.B; pidx += gridDim.x) {
        const uint32_t t = (uint32_t)(pidx / H), w = (uint32_t)(pidx % H);
        const uint32_t f = a.tflags[t];
        if (!(f & TF_RAND_LAYER) || (f & TF_DESTAB_FRESH)) continue;
        const uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + (size_t)CW * n;
        slice_store_rm(a.rm + t * a.rm_stride, a.RS, a.Hr, H, w,
                       [&](uint32_t j) { return j < n ? qx[(size_t)w * n + j] : 0u; },
                       [&](uint32_t j) { return j < n ? qz[(size_t)w * n + j] : 0u; });
    }
}

// Full column-packed -> row-packed copy (used when a measurement layer comes
// first and the row-packed copy is stale).
__global__ void k_qm_to_rm(LArgs a) {
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW;
    const uint32_t w = blockIdx.x, t = blockIdx.y;
    if (w == 0 && threadIdx.x == 0) a.tflags[t] |= TF_DESTAB_FRESH;
    const uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + (size_t)CW * n;
    slice_store_rm(a.rm + t * a.rm_stride, a.RS, a.Hr, H, w,
                   [&](uint32_t j) { return j < n ? qx[(size_t)w * n + j] : 0u; },
                   [&](uint32_t j) { return j < n ? qz[(size_t)w * n + j] : 0u; });
}

// Row-packed -> column-packed for dirty slices.
__global__ void k_rm_to_qm(LArgs a) {
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW;
    const uint32_t w = blockIdx.x, t = blockIdx.y;
    uint8_t *dirty = a.dirty + (size_t)t * CW;
    if (!dirty[w]) return;
    uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + (size_t)CW * n;
    slice_load_rm(a.rm + t * a.rm_stride, a.RS, a.Hr, H, n, w,
                  [&](uint32_t j, uint32_t x, uint32_t z) {
                      qx[(size_t)w * n + j] = x;
                      qz[(size_t)w * n + j] = z;
                  });
    __syncthreads();
    if (threadIdx.x == 0) dirty[w] = 0;
}

// ---------------------------------------------------------------- measurement
// Measured columns of a layer's ops (x plane, all CW words) into the
// item-major scratch cols[item][CW].  Tiles of 8 words x 128 items: two lanes
// per item, each reading 4 consecutive words (from the column-packed copy, or
// the row-packed one for dirty slices) and storing them as one 16-byte half
// of the item's 32-byte segment, so a warp's stores fill whole sectors.
constexpr uint32_t GATHER_ITEMS = 128;
__global__ void __launch_bounds__(2 * GATHER_ITEMS) k_gather_cols(LArgs a, uint32_t layer_arg) {
    const uint32_t n = a.P.n, CW = a.P.CW;
    const uint32_t layer = layer_arg & ~DET_SKIPPED;
    const uint32_t wl = (layer_arg & DET_SKIPPED) ? a.P.H : CW;    // words gathered
    const uint32_t t = blockIdx.z;
    const Layer M = a.P.layers[layer];
    const uint32_t i = blockIdx.y * GATHER_ITEMS + (threadIdx.x >> 1);
    if (i >= M.count) return;
    const uint32_t w0 = 8 * blockIdx.x + 4 * (threadIdx.x & 1);
    if (w0 >= wl) return;
    const uint32_t q = a.P.mitems[M.first + i].q;
    const uint8_t *dirty = a.dirty + (size_t)t * CW;
    const uint32_t *qx = a.qm + t * a.qm_stride;
    const uint32_t *rm = a.rm + t * a.rm_stride;
    uint32_t *col = a.cols + t * a.cols_stride + (size_t)i * CW;
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t w = w0 + k;
        v[k] = w >= wl ? 0u : dirty[w] ? rm_col_word(rm, a.RS, a.Hr, w, q, false) : qx[(size_t)w * n + q];
    }
    if ((CW & 3u) == 0 && ((uintptr_t)col & 15u) == 0 && w0 + 4 <= wl) {
        *reinterpret_cast<uint4 *>(col + w0) = make_uint4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (w0 + k < wl) col[w0 + k] = v[k];
    }
}

// Sign of the product of the stabilizers selected by the destabilizer column
// `colK` (H words), computed by one warp.  For commuting rows P_1..P_k the
// power of i of the product taken in any fixed order is
//   2 sum r_b + sum_b popc(x_b & z_b) + 2 sum_{b<b'} popc(z_b & x_b') - popc(X & Z)
// with X = xor of x_b, Z = xor of z_b (the rows commute, so the order does not
// change the product); the product must be +-Z_q, so X = 0.  The selected rows
// are first listed in `scratch` (2H words); each lane then walks them for its
// own words, keeping the running xor of z in registers.  If more than 2H rows
// are selected, the running xors live in scratch instead.
__device__ int det_outcome_warp(const uint32_t *__restrict__ rm, uint32_t RS, uint32_t Hr, uint32_t H,
                                const uint32_t *__restrict__ r, const uint32_t *__restrict__ colK,
                                uint32_t q, uint32_t *__restrict__ scratch, int *err) {
    const int lane = threadIdx.x & 31;
    // list the stabilizer rows (partners of the set destabilizer bits)
    uint32_t nk = 0;
    for (uint32_t base = 0; base < H; base += 32) {
        const uint32_t w = base + lane;
        const uint32_t kw = w < H ? colK[w] : 0u;
        const uint32_t c = __popc(kw);
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        uint32_t pos = nk + x - c, m = kw;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            if (pos < 2 * H) scratch[pos] = 32 * H + 32 * w + b;
            pos++;
        }
        nk += __shfl_sync(FULL_MASK, x, 31);
    }
    __syncwarp();
    int acc = 0, rsum = 0;
    bool ok = true;
    if (nk <= 2 * H) {
        for (uint32_t e = lane; e < nk; e += 32) rsum += (int)rbit(r, scratch[e]);
        // each lane owns DW words per chunk and walks the listed rows, issuing
        // the loads of one row's DW words at once
        constexpr int DW = 6;
        for (uint32_t c0 = 0; c0 < H; c0 += 32 * DW) {
            uint32_t zp[DW], xp[DW];
#pragma unroll
            for (int k = 0; k < DW; k++) { zp[k] = 0u; xp[k] = 0u; }
            for (uint32_t e = 0; e < nk; e++) {
                const uint32_t *__restrict__ row = rm + (size_t)scratch[e] * RS;
                uint32_t xv[DW], zv[DW];
#pragma unroll
                for (int k = 0; k < DW; k++) {
                    const uint32_t c = c0 + 32 * k + lane;
                    xv[k] = c < H ? row[c] : 0u;
                    zv[k] = c < H ? row[Hr + c] : 0u;
                }
#pragma unroll
                for (int k = 0; k < DW; k++) {
                    acc += __popc(xv[k] & zv[k]) + 2 * __popc(xv[k] & zp[k]);
                    zp[k] ^= zv[k];
                    xp[k] ^= xv[k];
                }
            }
#pragma unroll
            for (int k = 0; k < DW; k++) {
                const uint32_t c = c0 + 32 * k + lane;
                if (c < H) {
                    const uint32_t wantz = (c == (q >> 5)) ? (1u << (q & 31)) : 0u;
                    ok &= (xp[k] == 0u) && (zp[k] == wantz);
                }
            }
        }
    } else {
        uint32_t *Zp = scratch, *Xp = scratch + H;
        for (uint32_t c = lane; c < H; c += 32) { Zp[c] = 0; Xp[c] = 0; }
        __syncwarp();
        for (uint32_t base = 0; base < H; base += 32) {
            uint32_t kw = (base + lane < H) ? colK[base + lane] : 0u;
            uint32_t m = __ballot_sync(FULL_MASK, kw != 0);
            while (m) {
                const int L = __ffs(m) - 1;
                m &= m - 1;
                uint32_t word = __shfl_sync(FULL_MASK, kw, L);
                const uint32_t u = base + L;
                while (word) {
                    const int b = __ffs(word) - 1;
                    word &= word - 1;
                    const uint32_t s = 32 * H + 32 * u + b;
                    const uint32_t *__restrict__ row = rm + (size_t)s * RS;
                    for (uint32_t c = lane; c < H; c += 32) {
                        const uint32_t x = row[c], z = row[Hr + c];
                        acc += __popc(x & z) + 2 * __popc(x & Zp[c]);
                        Zp[c] ^= z;
                        Xp[c] ^= x;
                    }
                    if (lane == 0) rsum += (int)rbit(r, s);
                }
            }
        }
        for (uint32_t c = lane; c < H; c += 32) {
            const uint32_t wantz = (c == (q >> 5)) ? (1u << (q & 31)) : 0u;
            ok &= (Xp[c] == 0u) && (Zp[c] == wantz);
        }
    }
    acc = __reduce_add_sync(FULL_MASK, acc);
    rsum = __reduce_add_sync(FULL_MASK, rsum);
    const int e = (acc + 2 * rsum) & 3;
    if (!__all_sync(FULL_MASK, ok)) set_err(err, DERR_BAD_PRODUCT);
    if (e & 1) set_err(err, DERR_ODD_PHASE);
    __syncwarp();
    return (e >> 1) & 1;
}

// The same outcome from a listed support: lst[0..nk) are the set destabilizer
// slots of the column (nk <= SUPCAP, in any order; the row product is the same
// in every order because stabilizer rows commute), each naming stabilizer row
// 32H + slot.  Each row is read whole, as 8-byte vectors (DET_NV per lane per
// plane: one round trip per row for H <= 64 * DET_NV words, 320 at DET_NV = 5,
// which covers d = 71); needs an 8-byte aligned rm and an even Hr.
constexpr int DET_NV = 5;
__device__ __forceinline__ int det_outcome_list(const uint32_t *__restrict__ rm, uint32_t RS, uint32_t Hr,
                                                uint32_t H, const uint32_t *__restrict__ r,
                                                const uint16_t *lst, uint32_t nk, uint32_t q, int *err) {
    const int lane = threadIdx.x & 31;
    int acc = 0, rsum = 0;
    bool ok = true;
    for (uint32_t e = lane; e < nk; e += 32) rsum += (int)rbit(r, 32 * H + lst[e]);
    const uint32_t H2 = (H + 1) >> 1;
    for (uint32_t v0 = 0; v0 < H2; v0 += 32 * DET_NV) {
        uint32_t zp[2 * DET_NV], xp[2 * DET_NV];
#pragma unroll
        for (int k = 0; k < 2 * DET_NV; k++) { zp[k] = 0u; xp[k] = 0u; }
        for (uint32_t e = 0; e < nk; e++) {
            const uint32_t *__restrict__ row = rm + (size_t)(32 * H + lst[e]) * RS;
            const uint2 *__restrict__ rx = reinterpret_cast<const uint2 *>(row);
            const uint2 *__restrict__ rz = reinterpret_cast<const uint2 *>(row + Hr);
            uint2 xv[DET_NV], zv[DET_NV];
#pragma unroll
            for (int k = 0; k < DET_NV; k++) {
                const uint32_t j = v0 + 32 * k + lane;
                xv[k] = j < H2 ? rx[j] : make_uint2(0u, 0u);
                zv[k] = j < H2 ? rz[j] : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int k = 0; k < DET_NV; k++) {
                const uint32_t w = 2 * (v0 + 32 * k + lane);
                // a word past H (row padding, odd H) takes no part
                const uint32_t x0 = xv[k].x, z0 = zv[k].x;
                const uint32_t x1 = w + 1 < H ? xv[k].y : 0u, z1 = w + 1 < H ? zv[k].y : 0u;
                acc += __popc(x0 & z0) + 2 * __popc(x0 & zp[2 * k]) + __popc(x1 & z1) +
                       2 * __popc(x1 & zp[2 * k + 1]);
                zp[2 * k] ^= z0;
                xp[2 * k] ^= x0;
                zp[2 * k + 1] ^= z1;
                xp[2 * k + 1] ^= x1;
            }
        }
#pragma unroll
        for (int k = 0; k < 2 * DET_NV; k++) {
            const uint32_t w = 2 * (v0 + 32 * (k >> 1) + lane) + (k & 1);
            if (w < H) {
                const uint32_t wantz = (w == (q >> 5)) ? (1u << (q & 31)) : 0u;
                ok &= (xp[k] == 0u) && (zp[k] == wantz);
            }
        }
    }
    acc = __reduce_add_sync(FULL_MASK, acc);
    rsum = __reduce_add_sync(FULL_MASK, rsum);
    const int e = (acc + 2 * rsum) & 3;
    if (!__all_sync(FULL_MASK, ok)) set_err(err, DERR_BAD_PRODUCT);
    if (e & 1) set_err(err, DERR_ODD_PHASE);
    __syncwarp();
    return (e >> 1) & 1;
}

__device__ __forceinline__ void count(const LArgs &a, int k, unsigned long long v) {
    if (a.stats && v) atomicAdd(&a.stats[k], v);
}

// Sign flips to apply once the layer's measurements are done: X after a reset
// whose outcome is 1 (Pauli 1), Z of a RESET_ERROR (Pauli 3).
__device__ __forceinline__ void push_flip(const LArgs &a, uint32_t t, uint32_t layer, uint32_t q, uint32_t P) {
    const uint32_t k = atomicAdd(&a.flip_cnt[(size_t)t * a.P.n_layers + layer], 1u);
    a.flips[t * 2 * a.m_stride + k] = q | (P << 30);
}

// Flips implied by an op's outcome (resets with outcome 1).
__device__ __forceinline__ void outcome_flips(const LArgs &a, uint32_t t, uint32_t layer, const MItem &m,
                                              uint32_t o) {
    if (o && (m.flags & (MF_RESET | MF_RESET_AFTER | MF_RESET_ERR))) push_flip(a, t, layer, m.q, 1u);
}

__device__ __forceinline__ void write_record(const LArgs &a, uint32_t t, uint32_t rec, uint32_t out) {
    if (rec != 0xffffffffu && out)
        atomicOr(&a.call->record[(unsigned long long)t * a.call->rec_stride + (rec >> 6)], 1ull << (rec & 63));
}

// One warp scans a measured column (CW words): pivot = first set row of the
// stabilizer half (as slot - 32H, ~0 if none), size = number of set rows, and
// when size <= SUPCAP the set rows (in no particular order) into sup[].
// Columns of a multiple of 4 words (16-byte aligned) are read as 16-byte
// vectors, NV4 per lane in flight (128 * NV4 words per batch: NV4 = 5 takes a
// d = 71 column, 632 words, in one round trip); others as words, 256 per
// batch.  sup may point to shared or global memory.
template <int NV4 = 4>
__device__ __forceinline__ void warp_column_scan(const uint32_t *col, uint32_t H, uint32_t CW,
                                                 uint32_t &piv, uint32_t &size, uint16_t *sup) {
    constexpr int VN = 4 * NV4 > 8 ? 4 * NV4 : 8;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0, pv = 0xffffffffu;
    // one batch: NV vectors of VW words per lane, word index of vector k, element e:
    // w = VW * (v0 + 32 k + lane) + e (increasing in k, then e, for a lane)
    auto batch = [&](const uint32_t (&v)[VN], uint32_t wbase, uint32_t stride_w, int nk, int vw) {
        uint32_t c = 0, mine = 0xffffffffu;
#pragma unroll
        for (int k = 0; k < nk; k++)
#pragma unroll
            for (int e = 0; e < vw; e++) {
                const uint32_t x = v[k * vw + e];
                c += __popc(x);
                const uint32_t w = wbase + stride_w * k + e;
                if (mine == 0xffffffffu && w >= H && x) mine = 32 * (w - H) + __ffs(x) - 1;
            }
        mine = __reduce_min_sync(FULL_MASK, mine);
        if (pv == 0xffffffffu) pv = mine;
        uint32_t xs = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, xs, o);
            if (lane >= o) xs += y;
        }
        uint32_t pos = base + xs - c;
#pragma unroll
        for (int k = 0; k < nk; k++)
#pragma unroll
            for (int e = 0; e < vw; e++) {
                uint32_t m = v[k * vw + e];
                const uint32_t w = wbase + stride_w * k + e;
                while (m && pos < SUPCAP) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    sup[pos++] = (uint16_t)(32 * w + b);
                }
            }
        base += __shfl_sync(FULL_MASK, xs, 31);
    };
    if ((CW & 3u) == 0 && ((uintptr_t)col & 15u) == 0) {
        const uint4 *c4 = reinterpret_cast<const uint4 *>(col);
        const uint32_t n4 = CW >> 2;
        for (uint32_t v0 = 0; v0 < n4; v0 += 32 * NV4) {
            uint32_t v[VN];
#pragma unroll
            for (int k = 0; k < NV4; k++) {
                const uint32_t j = v0 + 32 * k + lane;
                const uint4 q = j < n4 ? c4[j] : make_uint4(0u, 0u, 0u, 0u);
                v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
            }
            batch(v, 4 * (v0 + lane), 128, NV4, 4);
        }
    } else {
        for (uint32_t w0 = 0; w0 < CW; w0 += 256) {
            uint32_t v[VN];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const uint32_t w = w0 + 32 * k + lane;
                v[k] = w < CW ? col[w] : 0u;
            }
            batch(v, w0 + lane, 32, 8, 1);
        }
    }
    piv = pv;
    size = base;
}

constexpr int DET_WARPS = 4;
// The general product as an out-of-line call for k_meas_det, whose list
// path is kept at 56 registers (nine 4-warp CTAs per SM) by not inlining it.
__device__ __noinline__ int det_outcome_warp_ool(const uint32_t *__restrict__ rm, uint32_t RS, uint32_t Hr,
                                                 uint32_t H, const uint32_t *__restrict__ r,
                                                 const uint32_t *__restrict__ colK, uint32_t q,
                                                 uint32_t *__restrict__ scratch, int *err) {
    return det_outcome_warp(rm, RS, Hr, H, r, colK, q, scratch, err);
}
// shared words per warp of k_meas_det: the 2H-word scratch of the general
// product, at least SUPCAP 16-bit support entries
__host__ __device__ constexpr uint32_t det_smem_words(uint32_t H) { return 2 * H > SUPCAP / 2 ? 2 * H : SUPCAP / 2; }

__global__ void __launch_bounds__(DET_WARPS * 32, 9) k_meas_det(LArgs a, uint32_t layer_arg) {
    extern __shared__ uint32_t smem[];
    const uint32_t layer = layer_arg & ~DET_SKIPPED;
    const uint32_t H = a.P.H, CW = a.P.CW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = blockIdx.y;
    const Layer M = a.P.layers[layer];
    const uint32_t i = blockIdx.x * DET_WARPS + warp;
    if (i >= M.count) return;
    const MItem m = a.P.mitems[M.first + i];
    uint8_t *stat = a.mstat + t * a.m_stride, *out = a.mout + t * a.m_stride;
    if (m.flags & MF_RESET_ERR) {
        if (lane == 0) {
            const uint32_t u2 = noise_word(a.call->st, t, m.nl + 2);
            if ((unsigned long long)u2 < a.P.thr[m.np].t[1]) push_flip(a, t, layer, m.q, 3u);
        }
        const uint32_t u0 = noise_word(a.call->st, t, m.nl);
        if ((unsigned long long)u0 >= a.P.thr[m.np].t[0]) {
            if (lane == 0) { stat[i] = MS_SKIP; out[i] = 0; }
            return;
        }
    }
    const uint32_t *col = a.cols + t * a.cols_stride + (size_t)i * CW;
    uint32_t *scratch = smem + (size_t)warp * det_smem_words(H);
    uint16_t *lst = reinterpret_cast<uint16_t *>(scratch);
    // pivot (first stabilizer row of the column), column size and support
    // (into shared memory; copied out, for the random-measurement kernel, when
    // the op is random)
    uint32_t pv, csize;
    const size_t ci = t * a.m_stride + i;
    warp_column_scan<5>(col, H, (layer_arg & DET_SKIPPED) ? H : CW, pv, csize, lst);
    __syncwarp();
    if (pv != 0xffffffffu) {
        uint16_t *sup = a.msup + ci * SUPCAP;
        for (uint32_t e = lane; e < min(csize, SUPCAP); e += 32) sup[e] = lst[e];
        if (lane == 0) {
            stat[i] = MS_RANDOM;
            atomicOr(&a.tflags[t], TF_RAND_LAYER);
            a.mpiv[ci] = pv;
            a.mbsz[ci] = csize;
            a.mstale[ci] = 0;
            a.mxn[ci] = XS_UNKNOWN;
        }
        return;
    }
    // deterministic: the stabilizer half is empty, so csize = K, the number of
    // set destabilizer bits, and lst holds their slots when K <= SUPCAP
    if (a.stats && lane == 0) {
        count(a, DC_DET, 1);
        count(a, DC_SUM_K, csize);
    }
    const uint32_t *rm = a.rm + t * a.rm_stride;
    const int o = (csize <= SUPCAP && (a.Hr & 1u) == 0 && ((uintptr_t)rm & 7u) == 0)
                      ? det_outcome_list(rm, a.RS, a.Hr, H, a.r + (size_t)t * CW, lst, csize, m.q, a.err)
                      : det_outcome_warp_ool(rm, a.RS, a.Hr, H, a.r + (size_t)t * CW, col, m.q, scratch, a.err);
    if (lane == 0) {
        stat[i] = MS_DONE;
        out[i] = (uint8_t)o;
        write_record(a, t, m.rec, (uint32_t)o);
        outcome_flips(a, t, layer, m, (uint32_t)o);
    }
}

// Outcomes of the ops that became deterministic during k_meas_rand (one warp
// each), from the layer's final tableau.  Most layers have none, so a fixed
// grid of warps strides over the (tableau, op) pairs instead of one CTA per
// 8 ops of every tableau.
__global__ void __launch_bounds__(DET_WARPS * 32) k_meas_late(LArgs a, uint32_t layer) {
    extern __shared__ uint32_t smem[];
    const uint32_t H = a.P.H, CW = a.P.CW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Layer M = a.P.layers[layer];
    // the layer is done with its random measurements: k_destab_to_rm made the
    // destabilizer half current where it was not, and the flag is cleared
    if (blockIdx.x == 0)
        for (uint32_t t = threadIdx.x; t < a.B; t += blockDim.x)
            if (a.tflags[t] & TF_RAND_LAYER) a.tflags[t] = TF_DESTAB_FRESH;
    const unsigned long long total = (unsigned long long)M.count * a.B;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * DET_WARPS;
    for (unsigned long long idx = (unsigned long long)blockIdx.x * DET_WARPS + warp; idx < total; idx += nwarps) {
        const uint32_t t = (uint32_t)(idx / M.count), i = (uint32_t)(idx % M.count);
        uint8_t *stat = a.mstat + t * a.m_stride, *out = a.mout + t * a.m_stride;
        if (stat[i] != MS_DETLATE) continue;
        const MItem m = a.P.mitems[M.first + i];
        const uint32_t *col = a.cols + t * a.cols_stride + (size_t)i * CW;
        const int o = det_outcome_warp(a.rm + t * a.rm_stride, a.RS, a.Hr, H, a.r + (size_t)t * CW,
                                       col, m.q, smem + (size_t)warp * 2 * H, a.err);
        if (lane == 0) {
            stat[i] = MS_DONE;
            out[i] = (uint8_t)o;
            write_record(a, t, m.rec, (uint32_t)o);
            outcome_flips(a, t, layer, m, (uint32_t)o);
        }
        __syncwarp();
    }
}

// rowsum(s, p) on the row-packed copy by one warp: row s <- row p * row s
// with r_s from 2 r_s + 2 r_p + (power of i) mod 4 (Appendix B).  Each lane
// issues the loads of RSW words of both rows before using any of them.
constexpr int RSW = 5;
__device__ __forceinline__ void rowsum_warp(uint32_t *rm, uint32_t RS, uint32_t Hr, uint32_t H,
                                            uint32_t *r, uint32_t s, uint32_t p, int *err) {
    const int lane = threadIdx.x & 31;
    const uint32_t *rp = rm + (size_t)p * RS;
    uint32_t *rs = rm + (size_t)s * RS;
    const uint32_t rwords = lane == 0 ? ((r[s >> 5] >> (s & 31)) & 1u) | (((r[p >> 5] >> (p & 31)) & 1u) << 1) : 0u;
    int acc = 0;
    for (uint32_t c0 = 0; c0 < H; c0 += 32 * RSW) {
        uint32_t xp[RSW], zp[RSW], xs[RSW], zs[RSW];
#pragma unroll
        for (int k = 0; k < RSW; k++) {
            const uint32_t c = c0 + 32 * k + lane;
            const bool in = c < H;
            xp[k] = in ? rp[c] : 0u;
            zp[k] = in ? rp[Hr + c] : 0u;
            xs[k] = in ? rs[c] : 0u;
            zs[k] = in ? rs[Hr + c] : 0u;
        }
#pragma unroll
        for (int k = 0; k < RSW; k++) {
            const uint32_t c = c0 + 32 * k + lane;
            acc += phase_word(xp[k], zp[k], xs[k], zs[k]);
            if (c < H) {
                rs[c] = xs[k] ^ xp[k];
                rs[Hr + c] = zs[k] ^ zp[k];
            }
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);   // (keeps k_meas_rand spill-free)
    if (lane == 0) {
        const uint32_t r_s = rwords & 1u, r_p = rwords >> 1;
        const int e = (int)(2 * r_s + 2 * r_p) + acc;
        if (e & 1) set_err(err, DERR_ODD_PHASE);
        const uint32_t nr = (uint32_t)((e & 3) >> 1);
        if (nr != r_s) atomicXor(&r[s >> 5], 1u << (s & 31));
    }
}

// rowsum(s, p) restricted to the words where row p is nonzero (listed in
// `wl`, `nwl` entries): elsewhere row p contributes neither an XOR nor a power
// of i (phase_word(0, 0, x, z) = 0), so the result is the full rowsum's.
__device__ __forceinline__ void rowsum_warp_sparse(uint32_t *rm, uint32_t RS, uint32_t Hr, uint32_t *r,
                                                   uint32_t s, uint32_t p, const uint16_t *wl,
                                                   uint32_t nwl, int *err) {
    const int lane = threadIdx.x & 31;
    const uint32_t *rp = rm + (size_t)p * RS;
    uint32_t *rs = rm + (size_t)s * RS;
    const uint32_t rwords = lane == 0 ? ((r[s >> 5] >> (s & 31)) & 1u) | (((r[p >> 5] >> (p & 31)) & 1u) << 1) : 0u;
    const uint32_t c0 = lane < nwl ? wl[lane] : 0u, c1 = lane + 32 < nwl ? wl[lane + 32] : 0u;
    const bool in0 = lane < nwl, in1 = lane + 32 < nwl;
    const uint32_t xp0 = in0 ? rp[c0] : 0u, zp0 = in0 ? rp[Hr + c0] : 0u;
    const uint32_t xs0 = in0 ? rs[c0] : 0u, zs0 = in0 ? rs[Hr + c0] : 0u;
    const uint32_t xp1 = in1 ? rp[c1] : 0u, zp1 = in1 ? rp[Hr + c1] : 0u;
    const uint32_t xs1 = in1 ? rs[c1] : 0u, zs1 = in1 ? rs[Hr + c1] : 0u;
    int acc = phase_word(xp0, zp0, xs0, zs0) + phase_word(xp1, zp1, xs1, zs1);
    if (in0) { rs[c0] = xs0 ^ xp0; rs[Hr + c0] = zs0 ^ zp0; }
    if (in1) { rs[c1] = xs1 ^ xp1; rs[Hr + c1] = zs1 ^ zp1; }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);   // (keeps k_meas_rand spill-free)
    if (lane == 0) {
        const uint32_t r_s = rwords & 1u, r_p = rwords >> 1;
        const int e = (int)(2 * r_s + 2 * r_p) + acc;
        if (e & 1) set_err(err, DERR_ODD_PHASE);
        const uint32_t nr = (uint32_t)((e & 3) >> 1);
        if (nr != r_s) atomicXor(&r[s >> 5], 1u << (s & 31));
    }
}

constexpr int RAND_THREADS = 1024;
constexpr int RAND_WARPS = RAND_THREADS / 32;
constexpr uint32_t PCAP = WaveCaps::PCAP_MAX;
constexpr uint32_t WCAP = WaveCaps::WCAP_MAX;     // ops applied per wave
// Pending ops examined per wave.  A d = 71 surface code's final layer takes 70
// waves with 1024 and 82 with 512: its first ops in circuit order conflict with
// one another, so a short window holds few that can join a wave.  Only the
// window's 5 bytes per op scale with it; the wave's per-op arrays (51 bytes)
// scale with WCAP, which keeps the layout small enough for the L1 cache's share
// of each SM (a layout 29 KB larger measured 7 % slower).
constexpr uint32_t WIN = WaveCaps::WINDOW_MAX;
constexpr uint32_t PAIRCAP = WaveCaps::PAIRCAP_MAX;
constexpr uint32_t JCAP = WaveCaps::JCAP_MAX;
constexpr uint32_t HT = 4096;                 // row hash slots (> PAIRCAP: never full)
constexpr uint32_t PWS = 4;                   // pivot words staged in shared memory per wave op
constexpr uint32_t CKEYS = 32 * PWS;          // sort keys of one pass of a multi-pivot row
constexpr uint16_t NOPIV = 0xffffu;
constexpr uint32_t HEMPTY = 0xffffffffu;
constexpr uint32_t QMAP_SMEM_MAX = 16384;     // qubits whose item map fits shared memory
static_assert(PCAP <= 8 * RAND_THREADS, "pending-list compaction keeps 8 entries per thread");
static_assert(WIN <= RAND_THREADS && WCAP <= WIN, "one thread per window op");
static_assert(HT > PAIRCAP && (HT & (HT - 1)) == 0, "row hash larger than the pair list, power of two");

// k_meas_rand's dynamic shared memory: byte offsets of its blocks (rand_layout)
struct RandLayout {
    uint32_t sh, pend, wpiv, wbsz, wxn, sel, sr, pwn, pairs, nxt, hslot, dlist, hkey, htail, ents, spc, spx, spz,
        hcnt, wkeys, wlist, wacc, qmask, blocked, pmask, wq, qmap, stat, stale, r, total;
};

// The wave state's scalars in k_meas_rand's dynamic shared memory, read and
// written by every CTA of the cluster.
struct RandShared {
    uint32_t np, nsel, npair, nent, firstrand, nrand, nstale, cut, serial, nmulti, npw;
};
__host__ __device__ __forceinline__ uint32_t rl_take(uint32_t &o, uint32_t bytes) {
    const uint32_t at = o;
    o = (o + bytes + 15u) & ~15u;
    return at;
}
// The layout's blocks, 16-byte aligned.
__host__ __device__ __forceinline__ RandLayout rand_layout(uint32_t n, uint32_t H) {
    RandLayout L;
    uint32_t o = 0;
    const bool item_smem = n <= QMAP_SMEM_MAX;
    L.sh = rl_take(o, sizeof(RandShared));
    L.pend = rl_take(o, 2 * PCAP);
    L.wpiv = rl_take(o, 2 * WIN);
    L.wbsz = rl_take(o, 2 * WIN);
    L.wxn = rl_take(o, WIN);
    L.sel = rl_take(o, 2 * WCAP);
    L.sr = rl_take(o, WCAP);
    L.pwn = rl_take(o, 4 * WCAP);
    L.pairs = rl_take(o, 4 * PAIRCAP);
    L.nxt = rl_take(o, 2 * PAIRCAP);
    L.hslot = rl_take(o, 2 * PAIRCAP);
    L.dlist = rl_take(o, 2 * PAIRCAP);
    L.hkey = rl_take(o, 4 * HT);
    L.htail = rl_take(o, 4 * HT);
    L.hcnt = rl_take(o, 4 * HT);
    L.ents = rl_take(o, 4 * JCAP);
    L.spc = rl_take(o, 2 * WCAP * PWS);
    L.spx = rl_take(o, 4 * WCAP * PWS);
    L.spz = rl_take(o, 4 * WCAP * PWS);
    L.wkeys = rl_take(o, 4 * CKEYS * RAND_WARPS);
    L.wlist = rl_take(o, 2 * 32 * RAND_WARPS);
    L.wacc = rl_take(o, 4 * 32 * RAND_WARPS);
    L.qmask = rl_take(o, 8 * H);
    L.blocked = rl_take(o, 4 * H);
    L.pmask = rl_take(o, 4 * H);
    L.wq = rl_take(o, 4 * WCAP);
    L.qmap = rl_take(o, item_smem ? 2 * n : 0u);
    L.stat = rl_take(o, item_smem ? n : 0u);
    L.stale = rl_take(o, item_smem ? n : 0u);
    L.r = rl_take(o, 8 * H);
    L.total = o;
    return L;
}
size_t rand_smem(uint32_t n, uint32_t H) { return rand_layout(n, H).total; }

// Block-wide exclusive scan of one value per thread (1024 threads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *warp_tot, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? warp_tot[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;          // inclusive totals per warp
        if (lane == nw - 1) *total = w;
    }
    __syncthreads();
    const uint32_t off = warp ? warp_tot[warp - 1] : 0u;
    const uint32_t res = off + x - v;
    __syncthreads();
    return res;
}

// Ascending bitonic sort of nk (a power of two, 32..CKEYS) keys in shared
// memory by one warp.
__device__ __forceinline__ void warp_sort_keys(uint32_t *keys, uint32_t nk) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = 2; k <= nk; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = lane; t < nk / 2; t += 32) {
                // pair (i, l = i + j), i < l: t with a zero bit inserted at j (a power of two)
                const uint32_t i = ((t & ~(j - 1u)) << 1) | (t & (j - 1u)), l = i + j;
                const bool up = (i & k) == 0;
                const uint32_t a = keys[i], b = keys[l];
                if ((a > b) == up) {
                    keys[i] = b;
                    keys[l] = a;
                }
            }
            __syncwarp();
        }
}

// The random measurements of one measurement layer of one tableau (one
// cluster of CTAs),
// in waves.  Sequential CHP applies them one by one in circuit order (Sec. 2.4:
// pivot, rowsum of the pivot into every other row with an X or Y on the
// measured qubit, destabilizer copy, +-Z_a with a random sign).  Two of them,
// j before k, commute bit for bit as tableau operations when neither pivot row
// has an X or Y on the other's qubit; a wave applies at once every pending op
// that commutes in this sense with every earlier pending op.  Conflicts are
// read from each pending op's cached pivot-row X support over the layer's
// items (mxs), recomputed only when the op's measured column changed (mstale)
// or its pivot row did (row versions), so selection needs no pass over
// columns and a window of up to WIN pending ops costs the same as a small one.
//
// Per wave: (1) ordered list of pending random ops; (2) refresh of stale
// pivots, X supports and pivot word counts of the window; (3) selection: an
// op is blocked when an earlier window op conflicts with it; (4) work lists,
// a warp per wave op: the rowsum pairs (rows of the op's measured column,
// except its pivot and the destabilizer partners of the wave's pivots, which
// end as copies of their pivot rows) linked per row through a shared-memory
// hash, the pivot's nonzero words staged in shared memory, and the pending
// ops whose measured column changes; (5) a row that receives one pivot gets
// it from one thread (its few nonzero words loaded once); a row that receives
// several gets them from one warp, which sorts the (word, chain position)
// keys of the chain so that every word is loaded once and its pivots applied
// in chain order -- the same order for every word of the row, which keeps the
// sum of the powers of i exact; pivots that commute with the row give an even
// power per pair, so each pair flips the row's sign by (r_p + power / 2) mod 2.
// Column updates and row copies touch other data and run in the same phase.
// A chain holding a pivot with more than PWS nonzero words is applied by one
// warp with full or word-listed rowsums, before the row copies.
// Cluster: rank 0's shared memory holds the wave state (lists, hash, window);
// every rank's warps take items of each phase (cluster-wide thread and warp
// indices) through distributed shared memory, and phases end at cluster
// barriers (release/acquire, so global and shared writes of one phase are
// seen by every rank in the next).  The pending-list compaction runs on rank
// 0 alone; per-warp scratch, the qubit -> item map and the pending-qubit mask
// are each rank's own.
__global__ void __launch_bounds__(RAND_THREADS, 1) k_meas_rand(LArgs a, uint32_t layer) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint32_t s_wt[32], s_tot;                     // rank 0's block scans
    __shared__ uint32_t xcnt[2 * RAND_WARPS];                // X-support counts of the 16-lane groups
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW, RS = a.RS, Hr = a.Hr, H4 = Hr >> 2;
    // one cluster of CTAs per tableau: rank 0 holds the wave state in its
    // shared memory, and the threads of every rank work on it (through
    // distributed shared memory); per-warp scratch stays in each CTA's own
    const cg::cluster_group cl = cg::this_cluster();
    const uint32_t crank = cl.block_rank(), ncl = cl.num_blocks();
    // one cluster per tableau: a grid row of any other size would give a
    // tableau two leaders (checked before any rank touches another's memory;
    // every CTA sees the same sizes, so all leave together)
    if (ncl != gridDim.x) {
        if (threadIdx.x == 0 && blockIdx.x == 0) set_err(a.err, DERR_BOUNDS);
        return;
    }
    const uint32_t t = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t gtid = crank * blockDim.x + threadIdx.x, GT = ncl * blockDim.x;   // cluster-wide
    const uint32_t gwarp = crank * (uint32_t)nw + (uint32_t)warp, GW = ncl * (uint32_t)nw;
    const bool lead = crank == 0;
    const Layer M = a.P.layers[layer];
    const RandLayout Lo = rand_layout(n, H);
    const uint32_t pcap = a.caps.pcap, wcap = min(a.caps.wcap, WCAP), paircap = a.caps.paircap,
                   jcap = a.caps.jcap;
    const uint32_t wmax = max(1u, min(a.caps.window, WIN));
    uint8_t *const gstat = a.mstat + t * a.m_stride, *out = a.mout + t * a.m_stride;
    uint32_t *const cols = a.cols + t * a.cols_stride;
    uint32_t *const rm = a.rm + t * a.rm_stride;
    uint32_t *const gr = a.r + (size_t)t * CW;
    uint8_t *const dirty = a.dirty + (size_t)t * CW;
    uint32_t *const mpiv = a.mpiv + t * a.m_stride, *const mbsz = a.mbsz + t * a.m_stride;
    uint8_t *const gmstale = a.mstale + t * a.m_stride;
    uint16_t *const msup = a.msup + t * a.m_stride * SUPCAP;
    uint16_t *const mxs = a.mxs + t * a.m_stride * XSCAP;
    uint8_t *const mxn = a.mxn + t * a.m_stride;
    uint32_t *const mxver = a.mxver + t * a.m_stride;
    uint32_t *const rowver = a.rowver + (size_t)t * 32 * H;
    uint16_t *const pwl = a.pwl + (size_t)t * WCAP * PWCAP;
    const bool item_smem = n <= QMAP_SMEM_MAX;
    // every rank's first test reads a flag that no kernel changes while this
    // one runs (k_meas_det sets it when an op of the layer is random,
    // k_meas_late clears it), so all ranks leave together or none does (no
    // rank may leave while others can still reach rank 0's shared memory)
    if (!(a.tflags[t] & TF_RAND_LAYER)) return;
    if (gtid == 0) a.P.layer_rand[layer] = 1;    // the layer has a random op (for the host's skip list)
    cl.sync();                         // every rank has started: rank 0's shared memory is reachable
    unsigned char *const sm = lead ? smraw : static_cast<unsigned char *>(cl.map_shared_rank((void *)smraw, 0));
    RandShared *const S = reinterpret_cast<RandShared *>(sm + Lo.sh);
    uint16_t *const pend = (uint16_t *)(sm + Lo.pend);    // pending item indices, circuit order
    uint16_t *const wpiv = (uint16_t *)(sm + Lo.wpiv);    // window: pivot (slot - 32H) or NOPIV
    uint16_t *const wbsz = (uint16_t *)(sm + Lo.wbsz);    // window: |x-column support| (saturated)
    uint8_t *const wxn = sm + Lo.wxn;                     // window: X-support length / XS_OVER
    uint16_t *const sel = (uint16_t *)(sm + Lo.sel);      // wave: window positions
    uint8_t *const sr = sm + Lo.sr;                       // wave: pivot sign before the wave
    uint32_t *const pwn = (uint32_t *)(sm + Lo.pwn);      // wave: nonzero words of the pivot row
    uint32_t *const pairs = (uint32_t *)(sm + Lo.pairs);  // row | wave index << 16
    uint16_t *const nxt = (uint16_t *)(sm + Lo.nxt);      // next pair of the same row (0xffff ends)
    uint16_t *const hslot = (uint16_t *)(sm + Lo.hslot);  // hash slot of the pair's row
    uint16_t *const dlist = (uint16_t *)(sm + Lo.dlist);  // rows (first pairs) applied by warps
    uint32_t *const hkey = (uint32_t *)(sm + Lo.hkey);    // hash: row
    uint32_t *const htail = (uint32_t *)(sm + Lo.htail);  // hash: first pair of the row's chain
    uint32_t *const hcnt = (uint32_t *)(sm + Lo.hcnt);    // hash: pairs linked to the row
    uint32_t *const ents = (uint32_t *)(sm + Lo.ents);    // item | wave index << 16 | bp << 31
    uint16_t *const spc = (uint16_t *)(sm + Lo.spc);      // wave pivots' nonzero words: index,
    uint32_t *const spx = (uint32_t *)(sm + Lo.spx);      //   x word
    uint32_t *const spz = (uint32_t *)(sm + Lo.spz);      //   z word
    uint32_t *const wkeys = (uint32_t *)(smraw + Lo.wkeys) + warp * CKEYS;   // per warp: sort keys
    uint16_t *const wlist = (uint16_t *)(smraw + Lo.wlist) + warp * 32;      //   chain pairs of a pass
    int *const wacc = (int *)(smraw + Lo.wacc) + warp * 32;                 //   powers of i per pair
    uint32_t *const qmask = (uint32_t *)(sm + Lo.qmask);  // destabilizer partners of the wave's pivots
    uint32_t *const blocked = (uint32_t *)(sm + Lo.blocked);   // per item: an earlier window op conflicts
    // per qubit: its layer item is still random and in no wave yet, or became
    // deterministic during the layer (the items whose measured columns are kept
    // current); scans of pivot and destabilizer rows test only these bits.
    // Each rank keeps its own copy; an op's bit is cleared on every rank when
    // it joins a wave.
    uint32_t *const pmask = (uint32_t *)(smraw + Lo.pmask);
    uint32_t *const wq = (uint32_t *)(sm + Lo.wq);        // wave: measured qubit
    // qubit -> layer item (each rank's own copy when it fits shared memory)
    uint16_t *const qmap = item_smem ? (uint16_t *)(smraw + Lo.qmap) : a.qmap + (size_t)t * n;
    uint8_t *const stat = item_smem ? sm + Lo.stat : gstat;
    uint8_t *const mstale = item_smem ? sm + Lo.stale : gmstale;
    uint32_t *const r = (uint32_t *)(sm + Lo.r);          // sign column, copied back at the end

    for (uint32_t w = gtid; w < CW; w += GT) r[w] = gr[w];
    if (item_smem) {
        for (uint32_t q = threadIdx.x; q < n; q += blockDim.x) qmap[q] = 0xffffu;
        for (uint32_t i = gtid; i < M.count; i += GT) {
            stat[i] = gstat[i];
            mstale[i] = gmstale[i];
        }
    } else {
        for (uint32_t q = gtid; q < n; q += GT) qmap[q] = 0xffffu;
    }
    wacc[lane] = 0;
    if (lane < 2) xcnt[2 * warp + lane] = 0u;
    for (uint32_t w = threadIdx.x; w < H; w += blockDim.x) pmask[w] = 0u;
    cl.sync();
    for (uint32_t i = threadIdx.x; i < M.count; i += blockDim.x) {
        const uint32_t q = a.P.mitems[M.first + i].q;
        if (item_smem) qmap[q] = (uint16_t)i;
        if (gstat[i] == MS_RANDOM) atomicOr(&pmask[q >> 5], 1u << (q & 31));
    }
    if (!item_smem)
        for (uint32_t i = gtid; i < M.count; i += GT) qmap[a.P.mitems[M.first + i].q] = (uint16_t)i;
    cl.sync();

    unsigned long long tlast = clock64();
#define PHASE(k)                                                              \
    do {                                                                      \
        if (lead && threadIdx.x == 0 && a.stats) {                            \
            const unsigned long long now_ = clock64();                         \
            atomicAdd(&a.stats[DC_PHASE0 + (k)], now_ - tlast);               \
            tlast = now_;                                                     \
        }                                                                     \
    } while (0)
    // sub-step times of warp 0 inside a phase (instrumentation, profiling only)
    unsigned long long tstep = 0;
#define STEP_START()                                                          \
    do {                                                                      \
        if (lead && threadIdx.x == 0 && a.stats) tstep = clock64();            \
    } while (0)
#define STEP(slot)                                                            \
    do {                                                                      \
        if (lead && threadIdx.x == 0 && a.stats) {                            \
            const unsigned long long now_ = clock64();                         \
            atomicAdd(&a.stats[(slot)], now_ - tstep);                        \
            tstep = now_;                                                     \
        }                                                                     \
    } while (0)
    auto chain_first = [&](uint32_t e) { return htail[hslot[e]]; };
    // a pair's sign flip: its pivot's sign plus half its (even) power of i
    auto pair_flip = [&](uint32_t x, int acc) -> uint32_t {
        if (acc & 1) set_err(a.err, DERR_ODD_PHASE);
        return (sr[x] + (uint32_t)((acc & 3) >> 1)) & 1u;
    };

    bool full_scan = true;          // pending list rebuilt from all items (first wave, or overflow)
    // every wave resolves at least one op (the first pending random op always
    // qualifies), so 2*count+3 passes bound the loop; exceeding it is a bug
    const uint32_t glimit = min(2 * M.count + 3, a.caps.wave_limit);
    for (uint32_t guard = 0;; guard++) {
        if (guard >= glimit) {
            if (gtid == 0) set_err(a.err, DERR_BOUNDS);
            break;
        }
        // ---- (1) ordered list of pending random measurements (first pcap):
        // from all items on the first wave or after an overflow, else by
        // compacting the previous list (ops only ever leave it); rank 0 alone
        if (lead) {
            if (full_scan) {
                uint32_t cnt = 0;
                const uint32_t per = (M.count + blockDim.x - 1) / blockDim.x;
                const uint32_t i0 = threadIdx.x * per, i1 = min(M.count, i0 + per);
                for (uint32_t i = i0; i < i1; i++) cnt += stat[i] == MS_RANDOM;
                uint32_t off = block_excl_scan(cnt, s_wt, &s_tot);
                for (uint32_t i = i0; i < i1; i++)
                    if (stat[i] == MS_RANDOM) {
                        if (off < pcap) pend[off] = (uint16_t)i;
                        off++;
                    }
                full_scan = s_tot > pcap;
            } else {
                // each thread owns at most PCAP / RAND_THREADS = 8 entries
                const uint32_t np0 = S->np;
                const uint32_t per = (np0 + blockDim.x - 1) / blockDim.x;
                const uint32_t k0 = threadIdx.x * per, k1 = min(np0, k0 + per);
                uint16_t keep[8];
                uint32_t cnt = 0;
#pragma unroll
                for (uint32_t d = 0; d < 8; d++) {
                    const uint32_t k = k0 + d;
                    if (k < k1) {
                        const uint16_t i = pend[k];
                        if (stat[i] == MS_RANDOM) keep[cnt++] = i;
                    }
                }
                const uint32_t off = block_excl_scan(cnt, s_wt, &s_tot);   // syncs: all reads done
#pragma unroll
                for (uint32_t d = 0; d < 8; d++)
                    if (d < cnt) pend[off + d] = keep[d];
            }
            for (uint32_t h = threadIdx.x; h < HT; h += blockDim.x) {
                hkey[h] = HEMPTY;
                htail[h] = 0xffffffffu;
                hcnt[h] = 0u;
            }
            for (uint32_t w = threadIdx.x; w < CW; w += blockDim.x) qmask[w] = 0u;
            __syncthreads();
            if (threadIdx.x == 0) {
                S->np = min(s_tot, pcap);
                S->nsel = 0; S->npair = 0; S->nent = 0; S->nstale = 0;
                S->firstrand = 0xffffffffu; S->nrand = 0; S->cut = 0xffffffffu;
                S->serial = 0; S->nmulti = 0; S->npw = 0;
            }
            __syncthreads();
            // ---- (2) window: cached pivots and X supports, on rank 0 (at
            // most WIN ops).  Ops whose measured column changed are listed in
            // `pairs` (free until the work lists) for a column rescan; ops whose
            // pivot row changed (or is new) in `ents` for an X-support rescan.
            const uint32_t np0 = S->np;
            if (np0) {
                const uint32_t nl = min(np0, wmax);
                for (uint32_t k = threadIdx.x; k < nl; k += blockDim.x) {
                    const uint32_t i = pend[k];
                    if (mstale[i]) {
                        pairs[atomicAdd(&S->nstale, 1u)] = k;
                        continue;
                    }
                    const uint32_t pv = mpiv[i], bs = mbsz[i], xn = mxn[i], xv = mxver[i];
                    wpiv[k] = (uint16_t)pv;
                    wbsz[k] = (uint16_t)min(bs, 65535u);
                    wxn[k] = (uint8_t)xn;
                    if (xn == XS_UNKNOWN || rowver[pv] != xv) ents[atomicAdd(&S->nent, 1u)] = k;
                }
                for (uint32_t w = (pend[0] >> 5) + threadIdx.x; w <= (pend[nl - 1] >> 5); w += blockDim.x) blocked[w] = 0u;
            }
        }
        cl.sync();
        PHASE(0);
        PHASE(1);
        const uint32_t np = S->np;
        if (np == 0) break;
        const uint32_t nlook = min(np, wmax);
        const uint32_t wfirst = pend[0], wlast = pend[nlook - 1];
        // Column rescans (a warp each) and X supports of the pivot rows over the
        // layer's items (16 lanes per op, 16-byte vectors of the x plane), in
        // one phase: a warp whose rescan finds a new pivot computes its X
        // support next, with one half; ops listed by the window pass for an
        // X-support rescan alone go two per warp.
        {
            const uint32_t nst = S->nstale, nx0 = S->nent;
            const uint32_t sub = (uint32_t)lane >> 4, sl = (uint32_t)lane & 15u;
            auto xs_one = [&](bool act, uint32_t k, uint32_t i, uint32_t pv) {
                uint32_t ver = 0;
                if (act) {
                    ver = rowver[pv];
                    const uint4 *px4 = reinterpret_cast<const uint4 *>(rm + (size_t)(32 * H + pv) * RS);
                    for (uint32_t j0 = 0; j0 < H4; j0 += 16 * 6) {
                        uint4 v[6];
#pragma unroll
                        for (int kk = 0; kk < 6; kk++) {
                            const uint32_t j = j0 + 16 * kk + sl;
                            v[kk] = j < H4 ? px4[j] : make_uint4(0u, 0u, 0u, 0u);
                        }
#pragma unroll
                        for (int kk = 0; kk < 6; kk++) {
                            const uint32_t j = j0 + 16 * kk + sl;
                            const uint32_t xw[4] = {v[kk].x, v[kk].y, v[kk].z, v[kk].w};
#pragma unroll
                            for (int e = 0; e < 4; e++) {
                                uint32_t m = 4 * j + e < H ? xw[e] & pmask[4 * j + e] : 0u;
                                while (m) {
                                    const int b = __ffs(m) - 1;
                                    m &= m - 1;
                                    const uint32_t u = 32 * (4 * j + e) + b;
                                    const uint32_t jj = u < n ? qmap[u] : 0xffffu;
                                    if (jj == 0xffffu) continue;
                                    const uint32_t pos = atomicAdd(&xcnt[2 * warp + sub], 1u);
                                    if (pos < XSCAP) mxs[(size_t)i * XSCAP + pos] = (uint16_t)jj;
                                }
                            }
                        }
                    }
                }
                __syncwarp();
                if (act && sl == 0) {
                    const uint32_t c = xcnt[2 * warp + sub];
                    const uint8_t xn = c <= XSCAP ? (uint8_t)c : XS_OVER;
                    mxn[i] = xn;
                    mxver[i] = ver;
                    wxn[k] = xn;
                    xcnt[2 * warp + sub] = 0u;
                    count(a, DC_XS_RECOMP, 1);
                }
                __syncwarp();
            };
            for (uint32_t it = gwarp; it < nst + (nx0 + 1) / 2; it += GW) {
                if (it < nst) {
                    const uint32_t k = pairs[it], i = pend[k];
                    uint32_t pv, bs;
                    warp_column_scan<5>(cols + (size_t)i * CW, H, CW, pv, bs, msup + (size_t)i * SUPCAP);
                    if (lane == 0) {
                        mpiv[i] = pv;
                        mbsz[i] = bs;
                        mstale[i] = 0;
                        count(a, DC_PIV_RECOMP, 1);
                        wbsz[k] = (uint16_t)min(bs, 65535u);
                        if (pv == 0xffffffffu) {             // became deterministic
                            wpiv[k] = NOPIV;
                            stat[i] = MS_DETLATE;
                            count(a, DC_DET_NOW, 1);
                        } else {
                            wpiv[k] = (uint16_t)pv;
                        }
                    }
                    xs_one(sub == 0 && pv != 0xffffffffu, k, i, pv);
                } else {
                    const uint32_t x = 2 * (it - nst) + sub;
                    const bool act = x < nx0;
                    const uint32_t k = act ? ents[x] : 0u, i = act ? pend[k] : 0u;
                    xs_one(act, k, i, act ? wpiv[k] : 0u);
                }
            }
        }
        cl.sync();
        PHASE(2);
        PHASE(3);
        // ---- (3) selection: for every conflicting pair of window ops the
        // later one is blocked; an op whose X support overflowed its list
        // blocks every later op (and itself, unless it is the first)
        if (lead) {        // (rank 0: at most WIN window ops)
            // two threads per window op, each walking every other entry of its
            // X-support list
            for (uint32_t tt = threadIdx.x; tt < 2 * nlook; tt += blockDim.x) {
                const uint32_t k = tt >> 1, half = tt & 1u;
                if (wpiv[k] == NOPIV) continue;
                if (!half) {
                    atomicMin(&S->firstrand, k);
                    atomicAdd(&S->nrand, 1u);
                }
                const uint32_t i = pend[k], xn = wxn[k];
                if (xn == XS_OVER) {
                    if (!half) atomicMin(&S->cut, k);
                    continue;
                }
                const uint16_t *xl = mxs + (size_t)i * XSCAP;
                for (uint32_t e = half; e < xn; e += 2) {
                    const uint32_t j = xl[e];
                    if (j == i || j < wfirst || j > wlast || stat[j] != MS_RANDOM) continue;
                    const uint32_t late = max(i, j);
                    atomicOr(&blocked[late >> 5], 1u << (late & 31));
                }
            }
            __syncthreads();
            if (S->nrand != 0) {          // (otherwise the window became deterministic)
                if (threadIdx.x == 0) S->nent = 0;   // the X-support list is done with
                const uint32_t cut = S->cut, fr = S->firstrand;
                // one window op per thread (the window is at most WIN <=
                // RAND_THREADS ops).  A selectable op commutes with every earlier
                // pending op, so any subset of them is a wave (those left out
                // stay pending).  The wave takes them while their rowsum pairs
                // (at most the column size less the pivot row) fit the pair
                // list, so that only a wave whose first op alone overflows it
                // takes the serial path.
                const uint32_t k = threadIdx.x, i = k < nlook ? pend[k] : 0u;
                const bool ok = k < nlook && wpiv[k] != NOPIV && !((blocked[i >> 5] >> (i & 31)) & 1u) &&
                                !(k > cut || (k == cut && k != fr));
                const uint32_t wt = ok ? max(1u, (uint32_t)wbsz[k]) - 1u : 0u;
                const uint32_t before = ok ? atomicAdd(&S->npw, wt) : 0u;
                if (ok && (before == 0 || before + wt <= paircap)) {
                    const uint32_t idx = atomicAdd(&S->nsel, 1u);
                    if (idx < wcap) {
                        sel[idx] = (uint16_t)k;
                        pwn[idx] = 0u;
                        stat[i] = MS_WAVE;
                        atomicOr(&qmask[wpiv[k] >> 5], 1u << (wpiv[k] & 31));
                        // the op leaves every rank's pending-qubit mask
                        const uint32_t q = a.P.mitems[M.first + i].q;
                        for (uint32_t c = 0; c < ncl; c++)
                            atomicAnd(cl.map_shared_rank(pmask, c) + (q >> 5), ~(1u << (q & 31)));
                    }
                }
            }
        }
        cl.sync();
        if (S->nrand == 0) {             // cluster-uniform: the window became deterministic
            PHASE(4);
            continue;
        }
        PHASE(4);
        // ---- (4) work lists: a wave op's rows are split among W warps (32
        // 16-byte vectors of each row per warp and block); the op's first warp
        // also links its rowsum pairs (shared-memory atomics on rank 0's hash)
        const uint32_t nsel = min(S->nsel, wcap);
        const uint32_t W = max(1u, min(8u, (H4 + 31) / 32));
        for (uint32_t tk = gwarp; tk < nsel * W; tk += GW) {
            // tasks 0..nsel-1: each op's first part (with the pair linking, on
            // rank 0's warps for the first 32 ops); then the other parts
            const uint32_t x = tk < nsel ? tk : (tk - nsel) / (W - 1);
            const uint32_t part = tk < nsel ? 0u : 1u + (tk - nsel) % (W - 1);
            const bool first = part == 0;
            STEP_START();
            const uint32_t k = sel[x], i = pend[k];
            const uint32_t q = wpiv[k], p = 32 * H + q;
            // loads of this op that do not depend on the row scans, issued
            // first: its support list (two entries per lane) and its qubit
            const uint32_t nb = wbsz[k];
            const uint16_t *sp = msup + (size_t)i * SUPCAP;
            const uint32_t sup0 = first && nb <= SUPCAP && (uint32_t)lane < nb ? sp[lane] : 0u;
            const uint32_t sup1 = first && nb <= SUPCAP && (uint32_t)lane + 32 < nb ? sp[lane + 32] : 0u;
            const uint32_t mq = first && lane == 0 ? a.P.mitems[M.first + i].q : 0u;
            // pending ops whose qubit has X or Y in row p or row q (their
            // measured columns change), and the nonzero words of row p: 16-byte
            // vectors of rows p (x, z) and q (x)
            const uint4 *px4 = reinterpret_cast<const uint4 *>(rm + (size_t)p * RS);
            const uint4 *pz4 = px4 + H4;
            const uint4 *qx4 = reinterpret_cast<const uint4 *>(rm + (size_t)q * RS);
            uint4 *rq4 = reinterpret_cast<uint4 *>(rm + (size_t)q * RS);
            for (uint32_t j0 = 32 * part; j0 < H4; j0 += 32 * W) {
                const uint32_t j = j0 + lane;
                const bool in = j < H4;
                const uint4 vx = in ? px4[j] : make_uint4(0u, 0u, 0u, 0u);
                const uint4 vz = in ? pz4[j] : make_uint4(0u, 0u, 0u, 0u);
                const uint4 vq = in ? qx4[j] : make_uint4(0u, 0u, 0u, 0u);
                // row q <- row p: no other op of the wave reads or writes row q
                // (it is no rowsum target), and each lane of each part stores
                // only the elements it has just read
                if (in) {
                    rq4[j] = vx;
                    rq4[H4 + j] = vz;
                }
                const uint32_t xw[4] = {vx.x, vx.y, vx.z, vx.w};
                const uint32_t zw[4] = {vz.x, vz.y, vz.z, vz.w};
                const uint32_t qw[4] = {vq.x, vq.y, vq.z, vq.w};
                uint32_t pmk[4];
#pragma unroll
                for (int e = 0; e < 4; e++) pmk[e] = 4 * j + e < H ? pmask[4 * j + e] : 0u;
                uint32_t mine = 0, ne = 0;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    mine += (xw[e] | zw[e]) != 0u;
                    ne += __popc((xw[e] | qw[e]) & pmk[e]);
                }
                if (__any_sync(FULL_MASK, ne != 0)) {
                    uint32_t ie = ne;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(FULL_MASK, ie, o);
                        if (lane >= o) ie += y;
                    }
                    uint32_t ebase = 0;
                    if (lane == 31) ebase = atomicAdd(&S->nent, ie);
                    ebase = __shfl_sync(FULL_MASK, ebase, 31) + ie - ne;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        uint32_t mm = ne ? ((xw[e] | qw[e]) & pmk[e]) : 0u;
                        while (mm) {
                            const int b = __ffs(mm) - 1;
                            mm &= mm - 1;
                            const uint32_t jj = qmap[32 * (4 * j + e) + b];
                            if (ebase < jcap) ents[ebase] = jj | (x << 16) | (((xw[e] >> b) & 1u) << 31);
                            ebase++;
                        }
                    }
                }
                // nonzero words of row p: placed after those the op's other
                // warps have counted (the list's order does not matter)
                if (__any_sync(FULL_MASK, mine != 0)) {
                    uint32_t incl = mine;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(FULL_MASK, incl, o);
                        if (lane >= o) incl += y;
                    }
                    uint32_t base = 0;
                    if (lane == 31) {
                        base = atomicAdd(&pwn[x], incl);
                        if (base + incl > PWS) S->serial = 1;
                    }
                    uint32_t pos = __shfl_sync(FULL_MASK, base, 31) + incl - mine;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        if ((xw[e] | zw[e]) == 0u) continue;
                        const uint32_t c = 4 * j + e;
                        if (pos < PWCAP) pwl[x * PWCAP + pos] = (uint16_t)c;
                        if (pos < PWS) {
                            spc[x * PWS + pos] = (uint16_t)c;
                            spx[x * PWS + pos] = xw[e];
                            spz[x * PWS + pos] = zw[e];
                        }
                        pos++;
                    }
                }
            }
            if (first && lane == 0) {
                sr[x] = (uint8_t)rbit(r, p);
                wq[x] = mq;
                // row q's sign is the pivot's (read by no other op of the wave)
                if (sr[x]) atomicOr(&r[q >> 5], 1u << (q & 31));
                else atomicAnd(&r[q >> 5], ~(1u << (q & 31)));
                dirty[p >> 5] = 1;
                dirty[q >> 5] = 1;
            }
            STEP(DC_W0_LIST_SCAN);
            if (!first) continue;       // (the op's rowsum pairs: its first warp)
            // rowsum pairs: rows of the measured column except the pivot and
            // the wave's destabilizer partners, linked per row
            // link pair f (row, this wave op) into its row's chain
            auto link_pair = [&](uint32_t f, uint32_t row) {
                if (f >= paircap) return;
                pairs[f] = row | (x << 16);
                uint32_t h = (row * 2654435761u) >> 20;       // HT = 4096 slots
                uint32_t probe = 0;
                for (; probe < HT; probe++) {
                    const uint32_t old = atomicCAS(&hkey[h], HEMPTY, row);
                    if (old == HEMPTY || old == row) break;
                    h = (h + 1) & (HT - 1);
                }
                if (probe == HT) {                   // cannot happen: HT > paircap
                    set_err(a.err, DERR_BOUNDS);
                    nxt[f] = 0xffffu;
                    hslot[f] = 0;
                    return;
                }
                const uint32_t prev = atomicExch(&htail[h], f);
                nxt[f] = prev == 0xffffffffu ? (uint16_t)0xffffu : (uint16_t)prev;
                hslot[f] = (uint16_t)h;
                // a row's second pair lists it for a warp (by hash slot)
                if (atomicAdd(&hcnt[h], 1u) == 1u) dlist[atomicAdd(&S->nmulti, 1u)] = (uint16_t)h;
            };
            if (nb <= SUPCAP) {
                // one append per warp and batch (a single shared counter would
                // otherwise take every lane's atomic in turn)
                for (uint32_t e0 = 0; e0 < nb; e0 += 32) {
                    const uint32_t e = e0 + lane;
                    const uint32_t row = e0 == 0 ? sup0 : sup1;
                    if (e < nb) dirty[row >> 5] = 1;
                    const bool keep = e < nb && row != p && !((qmask[row >> 5] >> (row & 31)) & 1u);
                    const uint32_t bal = __ballot_sync(FULL_MASK, keep);
                    uint32_t base = 0;
                    if (lane == 0 && bal) base = atomicAdd(&S->npair, (uint32_t)__popc(bal));
                    base = __shfl_sync(FULL_MASK, base, 0);
                    if (keep) link_pair(base + __popc(bal & ((1u << lane) - 1u)), row);
                }
            } else {
                const uint32_t *col = cols + (size_t)i * CW;
                for (uint32_t w = lane; w < CW; w += 32) {
                    uint32_t m = col[w];
                    if (m) dirty[w] = 1;
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        const uint32_t row = 32 * w + b;
                        if (row == p || ((qmask[row >> 5] >> (row & 31)) & 1u)) continue;
                        link_pair(atomicAdd(&S->npair, 1u), row);
                    }
                }
            }
            STEP(DC_W0_LIST_PAIRS);
        }
        cl.sync();
        PHASE(5);
        const uint32_t npair = S->npair, nent = S->nent;
        if (gtid == 0) {
            count(a, DC_WAVES, 1);
            count(a, DC_WAVE_OPS, nsel);
            count(a, DC_SUM_A, npair);
            count(a, DC_ROWSUM_PASSES, 1);
        }
        // serial: a dense pivot, or an overflowed list whose fallback reads
        // pivot rows from the tableau -- the row copies wait for them
        const bool serial = S->serial || npair > paircap || nent > jcap;
        if (gtid == 0) {
            count(a, DC_SERIAL_WAVES, serial ? 1u : 0u);
            count(a, DC_DENSE_WAVES, S->serial ? 1u : 0u);
        }
        // pivot rows become +-Z_a (16-byte stores over the Hr-word rows; the
        // words past H are zero in every row), with the coin as sign, and the
        // outcome; row q already holds the old pivot row (work lists)
        auto row_copies = [&](uint32_t st) {
            const uint32_t per = 2 * H4, tot = nsel * per;
            for (uint32_t tt = st; tt < tot; tt += GT) {
                const uint32_t x = tt / per, c = tt % per, p = 32 * H + wpiv[sel[x]], mq = wq[x];
                uint4 z = make_uint4(0u, 0u, 0u, 0u);
                if (c == H4 + (mq >> 7)) {
                    const uint32_t za = 1u << (mq & 31), zsub = (mq >> 5) & 3u;
                    z = make_uint4(zsub == 0 ? za : 0u, zsub == 1 ? za : 0u, zsub == 2 ? za : 0u, zsub == 3 ? za : 0u);
                }
                reinterpret_cast<uint4 *>(rm + (size_t)p * RS)[c] = z;
            }
            // sign, outcome, record, pending mask: a thread per wave op
            for (uint32_t x = st; x < nsel; x += GT) {
                const uint32_t k = sel[x], i = pend[k], q = wpiv[k], p = 32 * H + q;
                const MItem m = a.P.mitems[M.first + i];
                const uint32_t coin = (m.flags & MF_RESET_ERR) ? (noise_word(a.call->st, t, m.nl + 1) & 1u)
                                                               : coin_bit(a.call->st, t, m.coin);
                if (coin) atomicOr(&r[p >> 5], 1u << (p & 31));
                else atomicAnd(&r[p >> 5], ~(1u << (p & 31)));
                rowver[q]++;
                out[i] = (uint8_t)coin;
                stat[i] = MS_DONE;
                write_record(a, t, m.rec, coin);
                outcome_flips(a, t, layer, m, coin);
            }
        };
        auto singles = [&](uint32_t st) {
            // ---- (5a) rows with one pivot: a thread each; the others listed for warps
            if (npair <= paircap) {
                for (uint32_t e = st; e < npair; e += GT) {
                    const uint32_t f0 = chain_first(e);
                    const uint32_t x = pairs[e] >> 16, row = pairs[e] & 0xffffu;
                    const uint32_t nwd = pwn[x];
                    if (f0 != e || nxt[e] != 0xffffu) continue;     // a row of several pairs (listed when linked)
                    if (nwd > PWS) {                                 // one dense pivot (only in serial waves)
                        dlist[atomicAdd(&S->nmulti, 1u)] = (uint16_t)hslot[e];
                        continue;
                    }
                    uint32_t *rs = rm + (size_t)row * RS;
                    uint32_t xs[PWS], zs[PWS];
    #pragma unroll
                    for (uint32_t w = 0; w < PWS; w++) {
                        const bool o = w < nwd;
                        const uint32_t c = o ? spc[x * PWS + w] : 0u;
                        xs[w] = o ? rs[c] : 0u;
                        zs[w] = o ? rs[Hr + c] : 0u;
                    }
                    int acc = 0;
    #pragma unroll
                    for (uint32_t w = 0; w < PWS; w++) {
                        if (w >= nwd) continue;
                        const uint32_t c = spc[x * PWS + w], px_ = spx[x * PWS + w], pz_ = spz[x * PWS + w];
                        acc += phase_word(px_, pz_, xs[w], zs[w]);
                        rs[c] = xs[w] ^ px_;
                        rs[Hr + c] = zs[w] ^ pz_;
                    }
                    if (pair_flip(x, acc)) atomicXor(&r[row >> 5], 1u << (row & 31));
                    if (row >= 32 * H) atomicAdd(&rowver[row - 32 * H], 1u);
                }
            }
        };
        auto col_updates = [&](uint32_t gw) {
            // ---- (5b) measured columns of the remaining ops: x ^= x_{p,b} on the
            // pivot's column rows (not the pivot, not the wave's destabilizer
            // partners, which end as copies of their pivots); then row q's bit is
            // x_{p,b} and row p's is 0.  Touches no bit of another wave op's p or q.
            if (nent <= jcap) {
                // 8 lanes per listed update whose wave op has a listed support (at
                // most SUPCAP rows, 8 per lane loaded at once); larger columns by a
                // warp each below
                {
                    const uint32_t sub = (uint32_t)lane >> 3, sl = (uint32_t)lane & 7u;
                    for (uint32_t e0 = 4 * gw; e0 < nent; e0 += 4 * GW) {
                        const uint32_t e = e0 + sub;
                        const bool act = e < nent;
                        const uint32_t j = act ? ents[e] & 0xffffu : 0u, x = act ? (ents[e] >> 16) & 0x7fffu : 0u;
                        const uint32_t bp = act ? ents[e] >> 31 : 0u;
                        const uint32_t k = sel[x], q = wpiv[k], p = 32 * H + q;
                        if (!act || (bp && wbsz[k] > SUPCAP)) continue;
                        uint32_t *cj = cols + (size_t)j * CW;
                        if (bp) {
                            const uint16_t *sp = msup + (size_t)pend[k] * SUPCAP;
                            const uint32_t nb = wbsz[k];
                            uint32_t rows[SUPCAP / 8];
    #pragma unroll
                            for (uint32_t f = 0; f < SUPCAP / 8; f++) {
                                const uint32_t idx = sl + 8 * f;
                                rows[f] = idx < nb ? sp[idx] : 0xffffffffu;
                            }
                            // this lane's rows: every 8th of the list, in increasing
                            // word order, so rows of one word are often adjacent
                            uint32_t cw = 0xffffffffu, cm = 0u;
    #pragma unroll
                            for (uint32_t f = 0; f < SUPCAP / 8; f++) {
                                const uint32_t row = rows[f];
                                if (row == 0xffffffffu || row == p || ((qmask[row >> 5] >> (row & 31)) & 1u)) continue;
                                if ((row >> 5) != cw) {
                                    if (cm) atomicXor(&cj[cw], cm);
                                    cw = row >> 5;
                                    cm = 0u;
                                }
                                cm |= 1u << (row & 31);
                            }
                            if (cm) atomicXor(&cj[cw], cm);
                        }
                        if (sl == 0) {
                            if (bp) atomicOr(&cj[q >> 5], 1u << (q & 31));
                            else atomicAnd(&cj[q >> 5], ~(1u << (q & 31)));
                            atomicAnd(&cj[p >> 5], ~(1u << (p & 31)));
                            mstale[j] = 1;
                        }
                    }
                }
                for (uint32_t e = gw; e < nent; e += GW) {
                    const uint32_t j = ents[e] & 0xffffu, x = (ents[e] >> 16) & 0x7fffu, bp = ents[e] >> 31;
                    const uint32_t k = sel[x], q = wpiv[k], p = 32 * H + q;
                    if (!bp || wbsz[k] <= SUPCAP) continue;
                    uint32_t *cj = cols + (size_t)j * CW;
                    const uint32_t *col = cols + (size_t)pend[k] * CW;
                    for (uint32_t w = lane; w < CW; w += 32) {
                        uint32_t v = col[w] & ~qmask[w];
                        if (w == (p >> 5)) v &= ~(1u << (p & 31));
                        if (v) atomicXor(&cj[w], v);
                    }
                    if (lane == 0) {
                        atomicOr(&cj[q >> 5], 1u << (q & 31));
                        atomicAnd(&cj[p >> 5], ~(1u << (p & 31)));
                        mstale[j] = 1;
                    }
                }
            } else {
                // list overflow: every remaining op's column from the wave's columns
                // and the (not yet overwritten) pivot rows
                for (uint32_t j = gw; j < M.count; j += GW) {
                    if (stat[j] != MS_RANDOM && stat[j] != MS_DETLATE) continue;
                    uint32_t *cj = cols + (size_t)j * CW;
                    const uint32_t qb = a.P.mitems[M.first + j].q;
                    for (uint32_t x = 0; x < nsel; x++) {
                        const uint32_t k = sel[x], q = wpiv[k], p = 32 * H + q;
                        const uint32_t bp = (rm[(size_t)p * RS + (qb >> 5)] >> (qb & 31)) & 1u;
                        if (bp) {
                            const uint32_t *col = cols + (size_t)pend[k] * CW;
                            for (uint32_t w = lane; w < CW; w += 32) {
                                uint32_t v = col[w] & ~qmask[w];
                                if (w == (p >> 5)) v &= ~(1u << (p & 31));
                                cj[w] ^= v;
                            }
                        }
                        __syncwarp();
                        if (lane == 0) {
                            const uint32_t bq = (cj[q >> 5] >> (q & 31)) & 1u;
                            if (bp != bq) cj[q >> 5] ^= 1u << (q & 31);
                            cj[p >> 5] &= ~(1u << (p & 31));
                        }
                        __syncwarp();
                    }
                    if (lane == 0) mstale[j] = 1;
                }
            }
        };
        auto multi_rows = [&]() {
            // ---- (5c) rows with several pivots (or a dense one): a warp each
            if (npair <= paircap) {
                const uint32_t nm = S->nmulti;
                for (uint32_t d = gwarp; d < nm; d += GW) {
                    const uint32_t e0 = htail[dlist[d]], row = pairs[e0] & 0xffffu;
                    bool dense = false;                  // (only serial waves hold dense pivots)
                    if (serial)
                        for (uint32_t f = e0, it_ = 0; f < PAIRCAP && it_ < PAIRCAP; f = nxt[f], it_++)
                            dense |= pwn[pairs[f] >> 16] > PWS;
                    if (dense) {
                        // pivots in chain order with warp rowsums (signs set inside;
                        // pivot rows unchanged: the copies come after in this case)
                        for (uint32_t f = e0, it_ = 0; f < PAIRCAP && it_ < PAIRCAP; f = nxt[f], it_++) {
                            const uint32_t x = pairs[f] >> 16, p = 32 * H + wpiv[sel[x]];
                            if (pwn[x] <= PWCAP) rowsum_warp_sparse(rm, RS, Hr, r, row, p, pwl + x * PWCAP, pwn[x], a.err);
                            else rowsum_warp(rm, RS, Hr, H, r, row, p, a.err);
                            __syncwarp();
                        }
                        if (lane == 0 && row >= 32 * H) atomicAdd(&rowver[row - 32 * H], 1u);
                        continue;
                    }
                    uint32_t *rs = rm + (size_t)row * RS;
                    uint32_t cur = e0, flips = 0;
                    STEP_START();
                    for (uint32_t pass = 0; cur < PAIRCAP && pass < PAIRCAP; pass++) {
                        // up to 32 pairs of the chain, in chain order
                        uint32_t cnt = 0;
                        if (lane == 0) {
                            while (cur < PAIRCAP && cnt < 32) {
                                wlist[cnt++] = (uint16_t)cur;
                                cur = nxt[cur];
                            }
                        }
                        cur = __shfl_sync(FULL_MASK, cur, 0);
                        cnt = __shfl_sync(FULL_MASK, cnt, 0);
                        __syncwarp();
                        // sort keys (word, chain position, word slot)
                        uint32_t nk = 32;
                        while (nk < PWS * cnt) nk <<= 1;
                        const uint32_t lx = (uint32_t)lane < cnt ? pairs[wlist[lane]] >> 16 : 0u;
                        const uint32_t lnw = (uint32_t)lane < cnt ? pwn[lx] : 0u;
                        for (uint32_t idx = lane; idx < nk; idx += 32) wkeys[idx] = 0xffffffffu;
                        __syncwarp();
    #pragma unroll
                        for (uint32_t w = 0; w < PWS; w++)
                            if (w < lnw) wkeys[PWS * lane + w] = ((uint32_t)spc[lx * PWS + w] << 7) | ((uint32_t)lane << 2) | w;
                        __syncwarp();
                        STEP(DC_W0_MULTI_WALK);
                        warp_sort_keys(wkeys, nk);
                        STEP(DC_W0_MULTI_SORT);
                        // the sorted keys, 32 at a time: a segmented XOR prefix scan
                        // over each word's keys (chain order) gives every pivot the
                        // row word it meets, so all phases are computed at once;
                        // a word's last key stores the word (carries run across rows)
                        uint32_t carry_c = 0xffffffffu, carry_x = 0u, carry_z = 0u;
                        uint32_t pre_x[CKEYS / 32], pre_z[CKEYS / 32];      // row words, loaded at once
    #pragma unroll
                        for (uint32_t rr = 0; rr < CKEYS / 32; rr++) {
                            const uint32_t key = 32 * rr < nk ? wkeys[32 * rr + lane] : 0xffffffffu;
                            pre_x[rr] = key != 0xffffffffu ? rs[key >> 7] : 0u;
                            pre_z[rr] = key != 0xffffffffu ? rs[Hr + (key >> 7)] : 0u;
                        }
    #pragma unroll
                        for (uint32_t rr = 0; rr < CKEYS / 32; rr++) {
                            const uint32_t r0 = 32 * rr;
                            if (r0 >= nk) break;
                            const uint32_t key = wkeys[r0 + lane];
                            const bool valid = key != 0xffffffffu;
                            const uint32_t c = valid ? key >> 7 : 0xffffffffu;
                            const uint32_t ml = (key >> 2) & 31u, ms = key & 3u;
                            uint32_t px_ = 0u, pz_ = 0u;
                            const uint32_t sx = pre_x[rr], sz = pre_z[rr];
                            if (valid) {
                                const uint32_t gx = pairs[wlist[ml]] >> 16;
                                px_ = spx[gx * PWS + ms];
                                pz_ = spz[gx * PWS + ms];
                            }
                            const uint32_t cprev = __shfl_up_sync(FULL_MASK, c, 1);
                            const uint32_t cnext = __shfl_down_sync(FULL_MASK, c, 1);
                            bool head = lane == 0 ? c != carry_c : c != cprev;
                            uint32_t ix = px_, iz = pz_;
                            bool hacc = head;
                            for (int o = 1; o < 32; o <<= 1) {
                                const uint32_t yx = __shfl_up_sync(FULL_MASK, ix, o);
                                const uint32_t yz = __shfl_up_sync(FULL_MASK, iz, o);
                                const bool yh = __shfl_up_sync(FULL_MASK, hacc, o);
                                if (lane >= o && !hacc) {
                                    ix ^= yx;
                                    iz ^= yz;
                                    hacc = yh;
                                }
                            }
                            if (!hacc) {               // segment continues from the previous row
                                ix ^= carry_x;
                                iz ^= carry_z;
                            }
                            if (valid) {
                                const uint32_t rx = sx ^ ix ^ px_, rz = sz ^ iz ^ pz_;   // row word before this pivot
                                atomicAdd(&wacc[ml], phase_word(px_, pz_, rx, rz));
                                const bool last = lane == 31 ? (r0 + 32 >= nk || (wkeys[r0 + 32] >> 7) != c) : cnext != c;
                                if (last) {
                                    rs[c] = sx ^ ix;
                                    rs[Hr + c] = sz ^ iz;
                                }
                            }
                            carry_c = __shfl_sync(FULL_MASK, c, 31);
                            carry_x = __shfl_sync(FULL_MASK, ix, 31);
                            carry_z = __shfl_sync(FULL_MASK, iz, 31);
                            __syncwarp();
                        }
                        __syncwarp();
                        STEP(DC_W0_MULTI_ROWS);
                        if ((uint32_t)lane < cnt) {
                            flips ^= pair_flip(lx, wacc[lane]);
                            wacc[lane] = 0;
                        }
                        __syncwarp();
                    }
                    flips = __reduce_xor_sync(FULL_MASK, flips);
                    if (lane == 0) {
                        if (flips) atomicXor(&r[row >> 5], 1u << (row & 31));
                        if (row >= 32 * H) atomicAdd(&rowver[row - 32 * H], 1u);
                    }
                }
            } else {
                // pair-list overflow: one warp applies the pivots row by row, in wave order
                for (uint32_t w = gwarp; w < CW; w += GW) {
                    for (uint32_t x = 0; x < nsel; x++) {
                        const uint32_t k = sel[x], q = wpiv[k], p = 32 * H + q;
                        uint32_t m = cols[(size_t)pend[k] * CW + w] & ~qmask[w];
                        if (w == (p >> 5)) m &= ~(1u << (p & 31));
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1;
                            const uint32_t row = 32 * w + b;
                            rowsum_warp(rm, RS, Hr, H, r, row, p, a.err);
                            __syncwarp();
                            if (lane == 0 && row >= 32 * H) rowver[row - 32 * H]++;
                        }
                    }
                }
            }
        };
        // A wave without a dense pivot applies everything in one phase: rank
        // 0's warps take the rows of several pivots (its shared memory holds
        // their chains), the other ranks' threads the single-pivot rows, the
        // column updates and the row copies (the multi-pivot rows read the
        // staged pivot words, not the pivot rows the copies overwrite).  A
        // serial wave applies the rows of several pivots, and the dense ones,
        // after the single ones, then the row copies.
        if (!serial) {
            multi_rows();
            singles(GT - 1 - gtid);
            col_updates(GW - 1 - gwarp);
            row_copies(GT - 1 - gtid);
            cl.sync();
            PHASE(6);
            PHASE(7);
        } else {
            singles(gtid);
            col_updates(gwarp);
            cl.sync();
            PHASE(6);
            multi_rows();
            cl.sync();
            row_copies(gtid);
            cl.sync();
            PHASE(7);
        }
    }
#undef PHASE
#undef STEP
#undef STEP_START
    // after this barrier no rank reaches rank 0's shared memory again
    cl.sync();
    if (lead) {
        for (uint32_t w = threadIdx.x; w < CW; w += blockDim.x) gr[w] = r[w];
        if (item_smem)
            for (uint32_t i = threadIdx.x; i < M.count; i += blockDim.x) {
                gstat[i] = stat[i];
                gmstale[i] = mstale[i];
            }
    }
}

// X after resets with outcome 1 (r ^= z_a) and RESET_ERROR's Z (r ^= x_a),
// from the layer's flip list.
__global__ void k_cond(LArgs a, uint32_t layer) {
    __shared__ uint32_t sred[32];
    const uint32_t n = a.P.n, CW = a.P.CW;
    const uint32_t w = blockIdx.x, t = blockIdx.y;
    const uint32_t cnt = a.flip_cnt[(size_t)t * a.P.n_layers + layer];
    if (cnt == 0) return;
    const uint32_t *fl = a.flips + t * 2 * a.m_stride;
    const bool dty = a.dirty[(size_t)t * CW + w] != 0;
    const uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + (size_t)CW * n;
    const uint32_t *rm = a.rm + t * a.rm_stride;
    uint32_t v = 0;
    for (uint32_t e = threadIdx.x; e < cnt; e += blockDim.x) {
        const uint32_t f = fl[e], q = f & 0x3fffffffu, P = f >> 30;
        if (P == 1u) v ^= dty ? rm_col_word(rm, a.RS, a.Hr, w, q, true) : qz[(size_t)w * n + q];
        else v ^= dty ? rm_col_word(rm, a.RS, a.Hr, w, q, false) : qx[(size_t)w * n + q];
    }
    v = __reduce_xor_sync(FULL_MASK, v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t u = lane < nw ? sred[lane] : 0u;
        u = __reduce_xor_sync(FULL_MASK, u);
        if (lane == 0 && u) a.r[(size_t)t * CW + w] ^= u;
    }
}

// ---------------------------------------------------------------- host side
size_t layered_gate_smem(uint32_t n) { return (size_t)8 * ((n + 15u) & ~15u); }   // slots below round16(n)

size_t rand_smem(uint32_t n, uint32_t H);

int layered_supported(uint32_t n, const LaunchCfg &lc) {
    const uint32_t H = (n + 31) / 32;
    return layered_gate_smem(n) + 1024 <= lc.smem_optin && rand_smem(n, H) + 1024 <= lc.smem_optin;
}

size_t batch_bytes(uint32_t n, uint32_t count) {
    const size_t H = (n + 31) / 32, CW = 2 * H, Hr = round4((uint32_t)H), RS = 2 * Hr;
    size_t per = 4 * (2 * CW * (size_t)n + 64 * H * RS + CW) + CW + 4;
    return per * count + 1024;
}

// Lay out `count` tableaux of n qubits in the batch's allocation, reusing it
// when it is large enough (no cudaFree / cudaMalloc, so no device-wide
// synchronisation) and allocating a larger one otherwise.
int batch_alloc(Batch &b, uint32_t n, uint32_t count, std::string *err) {
    const size_t H = (n + 31) / 32, CW = 2 * H;
    const size_t Hr = round4((uint32_t)H), RS = 2 * Hr;
    const size_t qm_stride = 2 * CW * (size_t)n, rm_stride = 64 * H * RS;
    const size_t qm_b = 4 * qm_stride * count, rm_b = 4 * rm_stride * count;
    const size_t r_b = 4 * CW * count, d_b = CW * count, f_b = 4 * (size_t)count;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t need = up(qm_b) + up(rm_b) + up(r_b) + up(d_b) + up(f_b);
    if (!b.mem || b.cap < need) {
        batch_free(b);
        if (cudaMalloc(&b.mem, need) != cudaSuccess) {
            cudaGetLastError();
            b.mem = nullptr;
            *err = "cudaMalloc of " + std::to_string(need) + " bytes for tableaux failed";
            return STAB_ERR_OOM;
        }
        b.cap = need;
    }
    b.n = n;
    b.H = (uint32_t)H;
    b.CW = (uint32_t)CW;
    b.count = count;
    b.qm_stride = qm_stride;
    b.rm_stride = rm_stride;
    b.bytes = need;
    char *p = (char *)b.mem;
    b.qm = (uint32_t *)p; p += up(qm_b);
    b.rm = (uint32_t *)p; p += up(rm_b);
    b.r = (uint32_t *)p; p += up(r_b);
    b.dirty = (uint8_t *)p; p += up(d_b);
    b.tflags = (uint32_t *)p;
    b.rm_valid = false;
    return STAB_OK;
}

void batch_free(Batch &b) {
    if (b.mem) cudaFree(b.mem);
    b = Batch{};
}

static LArgs make_args(const HostProg *p, Batch &b, MeasScratch *ms, int *d_err) {
    // zeroed bytes, padding included: the graph cache compares LArgs byte for byte
    LArgs a;
    memset(static_cast<void *>(&a), 0, sizeof a);   // trivially copyable; its members are set below
    a.caps = g_caps;
    if (p) a.P = p->dev;
    a.P.n = b.n; a.P.H = b.H; a.P.CW = b.CW;
    a.qm = b.qm; a.qm_stride = b.qm_stride;
    a.rm = b.rm; a.rm_stride = b.rm_stride;
    a.Hr = round4(b.H); a.RS = 2 * a.Hr;
    a.r = b.r; a.dirty = b.dirty; a.tflags = b.tflags;
    if (ms && p) {
        a.cols = ms->cols;
        a.cols_stride = (unsigned long long)std::max<uint32_t>(1, p->dev.max_meas) * b.CW;
        a.mstat = ms->stat; a.mout = ms->out;
        a.m_stride = std::max<uint32_t>(1, p->dev.max_meas);
        a.mxs = ms->mxs;
        a.mxn = ms->mxn;
        a.mxver = ms->mxver;
        a.rowver = ms->rowver;
        a.qmap = ms->qmap;
        a.ev = ms->ev;
        a.ev_cnt = ms->ev_cnt;
        a.mpiv = ms->mpiv;
        a.mbsz = ms->mbsz;
        a.mstale = ms->mstale;
        a.msup = ms->msup;
        a.pwl = ms->pwl;
        a.flips = ms->flips;
        a.flip_cnt = ms->flip_cnt;
    }
    a.call = ms ? ms->call : nullptr;
    a.err = d_err;
    a.B = b.count;
    return a;
}

// Launch wrapper: counts the launch and, when the kind is selected, brackets
// it with CUDA events on its stream.
template <typename F>
static void launch(KernelProf *kp, uint32_t kind, cudaStream_t s, double bytes, F &&f) {
    if (!kp) { f(); return; }
    kp->launches++;
    if (kp->mask & (1u << kind)) {
        KernelProf::Rec r;
        kp->begin(kind, s, r);
        f();
        kp->end(r, s, bytes);
    } else {
        f();
    }
}

cudaError_t layered_init(Batch &b, cudaStream_t s, KernelProf *kp) {
    LArgs a = make_args(nullptr, b, nullptr, nullptr);
    launch(kp, STAB_KERNEL_OTHER, s, 0.0, [&] { k_init<<<1024, 256, 0, s>>>(a); });
    b.rm_valid = true;
    return cudaGetLastError();
}

cudaError_t layered_sync_qm(Batch &b, cudaStream_t s) {
    LArgs a = make_args(nullptr, b, nullptr, nullptr);
    k_rm_to_qm<<<dim3(b.CW, b.count), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Commutation of m Paulis with every row of one tableau (Sec. 3.2): row S
// anticommutes with P iff x_P . z_S + z_P . x_S is odd.  On the column-packed
// copy this is, for each 32-row slot word w, the XOR over the qubits j of
// z_j[w] where x_P has bit j and x_j[w] where z_P has bit j.  One warp per
// (Pauli, CT consecutive slot words); lanes stride over the qubits, so each
// load instruction reads 32 consecutive words of a [plane][word][qubit] row.
constexpr uint32_t CT = 4;
__global__ void __launch_bounds__(256) k_commute(const uint32_t *__restrict__ qx, uint32_t n, uint32_t H,
                                                 uint32_t CW, const unsigned long long *__restrict__ px,
                                                 const unsigned long long *__restrict__ pz, uint32_t m,
                                                 uint32_t *__restrict__ out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t ntile = (CW + CT - 1) / CT;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (warp >= (uint64_t)m * ntile) return;
    const uint32_t k = (uint32_t)(warp / ntile), w0 = (uint32_t)(warp % ntile) * CT;
    const uint32_t Wq = (n + 63) / 64;
    const uint32_t *qz = qx + (size_t)CW * n;
    const unsigned long long *xk = px + (size_t)k * Wq, *zk = pz + (size_t)k * Wq;
    uint32_t acc[CT];
#pragma unroll
    for (uint32_t t = 0; t < CT; t++) acc[t] = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const uint32_t xb = (uint32_t)(xk[j >> 6] >> (j & 63)) & 1u;
        const uint32_t zb = (uint32_t)(zk[j >> 6] >> (j & 63)) & 1u;
        if (!(xb | zb)) continue;
#pragma unroll
        for (uint32_t t = 0; t < CT; t++) {
            const uint32_t w = w0 + t;
            if (w >= CW) break;
            if (xb) acc[t] ^= qz[(size_t)w * n + j];
            if (zb) acc[t] ^= qx[(size_t)w * n + j];
        }
    }
#pragma unroll
    for (uint32_t t = 0; t < CT; t++)
        acc[t] = __reduce_xor_sync(FULL_MASK, acc[t]);
    if (lane != 0) return;
    // output: per Pauli [destabilizer half | stabilizer half], 2 Wq uint32 words each
    uint32_t *o = out + (size_t)k * 4 * Wq;
    const uint32_t tail = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xffffffffu;
#pragma unroll
    for (uint32_t t = 0; t < CT; t++) {
        const uint32_t w = w0 + t;
        if (w >= CW) break;
        const bool stab = w >= H;
        const uint32_t wh = stab ? w - H : w;
        uint32_t v = acc[t];
        if (wh == H - 1) v &= tail;
        o[(stab ? 2 * Wq : 0) + wh] = v;
        if (wh == H - 1 && H < 2 * Wq) o[(stab ? 2 * Wq : 0) + H] = 0;   // pad word of an odd H
    }
}

cudaError_t layered_commute(Batch &b, uint32_t index, const unsigned long long *px, const unsigned long long *pz,
                            size_t m, unsigned long long *out, cudaStream_t s, KernelProf *kp) {
    if (!m) return cudaSuccess;
    cudaError_t e = layered_sync_qm(b, s);
    if (e) return e;
    const uint64_t warps = (uint64_t)m * ((b.CW + CT - 1) / CT);
    const uint64_t blocks = (warps + 7) / 8;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    KernelProf::Rec rec;
    const bool timed = kp && (kp->mask & (1u << STAB_KERNEL_COMMUTE));
    if (kp) kp->launches++;
    // bytes per launch: the tableau's column-packed planes once, the Paulis, the output
    const double bytes = 8.0 * b.CW * b.n + 16.0 * m * ((b.n + 63) / 64) + 16.0 * m * ((b.n + 63) / 64);
    if (timed) kp->begin(STAB_KERNEL_COMMUTE, s, rec);
    k_commute<<<(unsigned)blocks, 256, 0, s>>>(b.qm + (size_t)index * b.qm_stride, b.n, b.H, b.CW, px, pz,
                                               (uint32_t)m, (uint32_t *)out);
    if (timed) kp->end(rec, s, bytes);
    return cudaGetLastError();
}

WaveCaps g_caps;

void set_wave_caps(const WaveCaps &c) {
    g_caps.pcap = std::max(1u, std::min(c.pcap, WaveCaps::PCAP_MAX));
    g_caps.wcap = std::max(1u, std::min(c.wcap, WaveCaps::WCAP_MAX));
    g_caps.paircap = std::min(c.paircap, WaveCaps::PAIRCAP_MAX);
    g_caps.jcap = std::min(c.jcap, WaveCaps::JCAP_MAX);
    g_caps.mark_budget = c.mark_budget;
    g_caps.window = std::max(1u, c.window);
    g_caps.wave_limit = std::max(1u, c.wave_limit);
}

static cudaError_t layered_issue(const HostProg &p, Batch &b, MeasScratch &ms, int *d_err,
                                 const LaunchCfg &lc, cudaStream_t s, KernelProf *kp,
                                 unsigned long long *d_stats, const uint8_t *skip);

int graph_slot_init(GraphSlot &g) {
    if (g.gs) return 0;
    if (cudaStreamCreateWithFlags(&g.gs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        graph_slot_free(g);
        return -1;
    }
    return 0;
}

void graph_slot_free(GraphSlot &g) {
    if (g.gs) cudaStreamDestroy(g.gs);
    if (g.in) cudaEventDestroy(g.in);
    if (g.out) cudaEventDestroy(g.out);
    g = GraphSlot{};
}

void prog_graphs_free(HostProg &p) {
    if (p.gdone) cudaEventSynchronize(p.gdone);
    if (p.gexec) cudaGraphExecDestroy(p.gexec);
    if (p.gdone) cudaEventDestroy(p.gdone);
    p.gexec = nullptr;
    p.gdone = nullptr;
    p.gkey.clear();
}

// Launch sequences longer than this are issued plainly instead of being
// captured as one graph: a program of tens of thousands of layers (the random
// n-wide benchmark at n = 2048 has 4.2 M ops) made capture crash the host
// process, while graphs of a few thousand nodes replay fine.
constexpr uint64_t GRAPH_MAX_NODES = 4096;
static uint64_t graph_nodes(const HostProg &p) {
    uint64_t k = 4;                                   // memsets, noise events
    for (const Run &R : p.runs) k += R.type == LT_GATE ? 1 : 7;
    return k;
}

// CTAs per tableau (cluster size) of k_meas_rand.  One or a few tableaux
// leave most SMs idle and are bound by one SM's issue rate and the latency of
// each wave's phases, so each tableau's waves are spread over a cluster of up
// to 8 SMs; a batch that fills the GPU with one CTA per tableau keeps one.
// STAB_RAND_CLUSTER (1..8) overrides.  A size the GPU cannot co-schedule with
// this shared-memory footprint (cudaOccupancyMaxActiveClusters == 0) is
// halved until it can.
static uint32_t rand_cluster_size(const LaunchCfg &lc, uint32_t count, size_t rsm) {
    static const int env = [] {
        const char *v = getenv("STAB_RAND_CLUSTER");
        const int k = v ? atoi(v) : 0;
        return k >= 1 && k <= 8 ? k : 0;
    }();
    uint32_t want = env ? (uint32_t)env
                        : (uint32_t)std::max(1, std::min(8, lc.sm_count / (int)std::max<uint32_t>(1, count)));
    static std::mutex mu;
    static std::map<std::tuple<int, uint32_t, size_t>, bool> fits;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    std::lock_guard<std::mutex> lk(mu);
    for (; want > 1; want >>= 1) {
        const auto key = std::make_tuple(dev, want, rsm);
        auto it = fits.find(key);
        if (it == fits.end()) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = want;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(want, 1, 1);
            cfg.blockDim = dim3(RAND_THREADS, 1, 1);
            cfg.dynamicSmemBytes = rsm;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            const cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, (const void *)k_meas_rand, &cfg);
            if (e) cudaGetLastError();
            it = fits.emplace(key, e == cudaSuccess && nc > 0).first;
        }
        if (it->second) break;
    }
    return want;
}

static cudaError_t launch_meas_rand(const LArgs &a, uint32_t layer, uint32_t count, uint32_t ncl, size_t rsm,
                                    cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ncl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ncl, count, 1);
    cfg.blockDim = dim3(RAND_THREADS, 1, 1);
    cfg.dynamicSmemBytes = rsm;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_meas_rand, a, layer);
}

static cudaError_t layered_run_seq(const HostProg &p, Batch &b, MeasScratch &ms, const DevStreams &st,
                                   unsigned long long *record, size_t rec_stride, int *d_err,
                                   const LaunchCfg &lc0, cudaStream_t s, KernelProf *kp,
                                   unsigned long long *d_stats, GraphSlot *gsl, const uint8_t *skip);

// A run of the program on the batch; `fresh`: the batch holds |0...0> tableaux
// (the runs whose random layers the circuit fixes, see HostProg::rand_learn).
cudaError_t layered_run(const HostProg &p, Batch &b, MeasScratch &ms, const DevStreams &st,
                        unsigned long long *record, size_t rec_stride, int *d_err,
                        const LaunchCfg &lc0, cudaStream_t s, KernelProf *kp,
                        unsigned long long *d_stats, GraphSlot *gsl, bool fresh) {
    HostProg &hp = const_cast<HostProg &>(p);
    const bool learn = fresh && hp.rand_learn;
    const uint32_t nl = (uint32_t)p.layers.size();
    if (learn && hp.rand_state == 1) {
        // the marks of an earlier run, once its read-back has landed
        const cudaError_t q = cudaEventQuery(hp.rand_ev);
        if (q == cudaSuccess) {
            int derr = 0;
            memcpy(&derr, hp.rand_host + nl, sizeof derr);
            if (derr == DERR_NONE) {
                hp.rand_skip.assign(nl, 0);
                for (uint32_t l = 0; l < nl; l++)
                    hp.rand_skip[l] = p.layers[l].type == LT_MEAS && !hp.rand_host[l];
                hp.rand_state = 2;
            } else {
                hp.rand_state = 0;       // learn again from a run without device errors
            }
        } else {
            cudaGetLastError();          // (not ready yet: clear the status)
        }
    }
    const uint8_t *skip = learn && hp.rand_state == 2 ? hp.rand_skip.data() : nullptr;
    cudaError_t e = layered_run_seq(p, b, ms, st, record, rec_stride, d_err, lc0, s, kp, d_stats, gsl, skip);
    if (!e && learn && hp.rand_state == 0) {
        // queue the read-back of this run's marks and of the device error flag
        if (!hp.rand_host && cudaMallocHost(&hp.rand_host, nl + sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            hp.rand_host = nullptr;
            return cudaSuccess;          // (no learning without the pinned buffer)
        }
        if (!hp.rand_ev && cudaEventCreateWithFlags(&hp.rand_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            hp.rand_ev = nullptr;
            return cudaSuccess;
        }
        e = cudaMemcpyAsync(hp.rand_host, p.dev.layer_rand, nl, cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaMemcpyAsync(hp.rand_host + nl, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaEventRecord(hp.rand_ev, s);
        if (!e) hp.rand_state = 1;
    }
    return e;
}

static cudaError_t layered_run_seq(const HostProg &p, Batch &b, MeasScratch &ms, const DevStreams &st,
                                   unsigned long long *record, size_t rec_stride, int *d_err,
                                   const LaunchCfg &lc0, cudaStream_t s, KernelProf *kp,
                                   unsigned long long *d_stats, GraphSlot *gsl, const uint8_t *skip) {
    {
        const int lim = (int)(lc0.smem_optin - 1024);
        smem_attr_once(0, (const void *)k_gate_run<true>, lim);
        smem_attr_once(4, (const void *)k_gate_run<false>, lim);
        smem_attr_once(1, (const void *)k_meas_det, lim);
        smem_attr_once(2, (const void *)k_meas_late, lim);
        smem_attr_once(3, (const void *)k_meas_rand, lim);
    }
    LaunchCfg lc = lc0;
    lc.rand_cluster = rand_cluster_size(lc0, b.count, rand_smem(b.n, b.H));
    // this call's inputs, read by the kernels from device memory (a pageable
    // source is staged before cudaMemcpyAsync returns)
    CallArgs ca{};
    ca.st = st;
    ca.record = record;
    ca.rec_stride = rec_stride;
    cudaError_t e = cudaMemcpyAsync(ms.call, &ca, sizeof ca, cudaMemcpyHostToDevice, s);
    if (e) return e;
    if (!gsl || !gsl->gs || (kp && kp->mask) || graph_nodes(p) > GRAPH_MAX_NODES)
        return layered_issue(p, b, ms, d_err, lc, s, kp, d_stats, skip);
    // Graph replay on the slot's stream, after the work already queued on s.
    // The captured sequence depends only on the kernel arguments (per-call
    // inputs excluded) and on whether the row-packed copy is valid on entry.
    HostProg &hp = const_cast<HostProg &>(p);
    LArgs ka = make_args(&p, b, &ms, d_err);
    ka.stats = nullptr;                  // (this path runs only with profiling off)
    std::vector<unsigned char> key(sizeof(LArgs) + 3);
    memcpy(key.data(), &ka, sizeof ka);
    key[sizeof ka] = b.rm_valid ? 1 : 0;
    key[sizeof ka + 1] = (unsigned char)lc.rand_cluster;
    key[sizeof ka + 2] = skip ? 1 : 0;
    if (!hp.gdone && cudaEventCreateWithFlags(&hp.gdone, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return layered_issue(p, b, ms, d_err, lc, s, kp, d_stats, skip);
    }
    e = cudaEventRecord(gsl->in, s);
    if (!e) e = cudaStreamWaitEvent(gsl->gs, gsl->in, 0);
    if (e) return e;
    if (hp.gexec && hp.gkey == key) {
        e = cudaGraphLaunch(hp.gexec, gsl->gs);
        if (kp) kp->launches += hp.glaunches;
        b.rm_valid = hp.grm_after;
    } else {
        e = cudaStreamBeginCapture(gsl->gs, cudaStreamCaptureModeThreadLocal);
        if (e) {
            // no capture on this stream: run the launches plainly on it instead
            cudaGetLastError();
            e = layered_issue(p, b, ms, d_err, lc, gsl->gs, kp, d_stats, skip);
            if (!e) e = cudaEventRecord(gsl->out, gsl->gs);
            if (!e) e = cudaStreamWaitEvent(s, gsl->out, 0);
            return e;
        }
        const unsigned long long n0 = kp ? kp->launches : 0;
        const cudaError_t ei = layered_issue(p, b, ms, d_err, lc, gsl->gs, kp, d_stats, skip);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(gsl->gs, &g);
        if (ei || ec) {
            if (g) cudaGraphDestroy(g);
            hp.gkey.clear();
            return ei ? ei : ec;
        }
        hp.glaunches = kp ? kp->launches - n0 : 0;
        hp.grm_after = b.rm_valid;
        // the executable graph is updated only after its last launch finished
        e = cudaEventSynchronize(hp.gdone);
        if (!e && hp.gexec && hp.gcl != lc.rand_cluster) {
            cudaGraphExecDestroy(hp.gexec);
            hp.gexec = nullptr;
        }
        if (!e && hp.gexec) {
            cudaGraphExecUpdateResultInfo info{};
            if (cudaGraphExecUpdate(hp.gexec, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(hp.gexec);
                hp.gexec = nullptr;
            }
        }
        if (!e && !hp.gexec) {
            e = cudaGraphInstantiate(&hp.gexec, g, 0);
            if (!e) hp.gcl = lc.rand_cluster;
        }
        cudaGraphDestroy(g);
        hp.gkey = e ? std::vector<unsigned char>() : key;
        if (!e) e = cudaGraphLaunch(hp.gexec, gsl->gs);
    }
    if (!e) e = cudaEventRecord(hp.gdone, gsl->gs);
    if (!e) e = cudaEventRecord(gsl->out, gsl->gs);
    if (!e) e = cudaStreamWaitEvent(s, gsl->out, 0);
    return e;
}

static cudaError_t layered_issue(const HostProg &p, Batch &b, MeasScratch &ms, int *d_err,
                                 const LaunchCfg &lc, cudaStream_t s, KernelProf *kp,
                                 unsigned long long *d_stats, const uint8_t *skip) {
    LArgs a = make_args(&p, b, &ms, d_err);
    a.stats = (kp && kp->mask) ? d_stats : nullptr;     // counters only while profiling
    const size_t rsm = rand_smem(b.n, b.H);
    cudaMemsetAsync(ms.flip_cnt, 0, sizeof(uint32_t) * std::max<size_t>(1, p.layers.size()) * b.count, s);
    if (p.dev.ev_total) {
        cudaMemsetAsync(ms.ev_cnt, 0, sizeof(uint32_t) * p.layers.size() * b.count, s);
        const unsigned long long work = (unsigned long long)p.dev.n_gitems * b.count;
        const uint32_t blocks = (uint32_t)std::min<unsigned long long>((work + 255) / 256, 8ull * lc.sm_count * 8);
        launch(kp, STAB_KERNEL_OTHER, s, 0.0, [&] { k_noise_events<<<blocks, 256, 0, s>>>(a); });
    }
    // Gate-run CTA size: one tableau's slices are few and large (two 1024-thread
    // CTAs per SM at d = 71); a batch's many small slices run best as 128-thread
    // CTAs, many per SM, so that layer barriers stall fewer warps at a time
    // (measured on GB300: d = 31 x 128 shots, gate runs 12.5 -> 8.9 ms).
    const uint32_t gthreads = b.count >= 2
        ? std::min<uint32_t>(128, std::max<uint32_t>(64, (p.dev.max_gitems / 2 + 31) / 32 * 32))
        : std::min<uint32_t>(1024, std::max<uint32_t>(64, (p.dev.max_gitems / 2 + 31) / 32 * 32));
    const size_t gsm = layered_gate_smem(b.n);
    int32_t cond_pending = -1;      // measurement layer whose flips the next gate run applies
    for (size_t k = 0; k < p.runs.size(); k++) {
        const Run &R = p.runs[k];
        if (R.type == LT_GATE) {
            GRun g{};
            g.l0 = R.l0; g.l1 = R.l1;
            g.cond_layer = cond_pending;
            cond_pending = -1;
            const bool next_meas = k + 1 < p.runs.size() && p.runs[k + 1].type == LT_MEAS;
            g.want_rm = next_meas ? 1u : 0u;
            launch(kp, STAB_KERNEL_GATE_RUN, s, R.alg_bytes * b.count,
                   [&] {
                       if (gthreads == 1024)
                           k_gate_run<true><<<dim3(b.CW, b.count), gthreads, gsm, s>>>(a, g);
                       else
                           k_gate_run<false><<<dim3(b.CW, b.count), gthreads, gsm, s>>>(a, g);
                   });
            b.rm_valid = next_meas;
        } else {
            const uint32_t l = R.l0;
            const Layer &L = p.layers[l];
            if (!b.rm_valid) {
                launch(kp, STAB_KERNEL_OTHER, s, 0.0,
                       [&] { k_qm_to_rm<<<dim3(b.CW, b.count), 256, 0, s>>>(a); });
                b.rm_valid = true;
            }
            const bool skipped = skip && skip[l];
            launch(kp, STAB_KERNEL_OTHER, s, 0.0, [&] {
                k_gather_cols<<<dim3(((skipped ? b.H : b.CW) + 7) / 8, (L.count + GATHER_ITEMS - 1) / GATHER_ITEMS,
                                     b.count),
                                2 * GATHER_ITEMS, 0, s>>>(a, skipped ? l | DET_SKIPPED : l);
            });
            const uint32_t nb = (L.count + DET_WARPS - 1) / DET_WARPS;
            launch(kp, STAB_KERNEL_MEAS_DET, s, 0.0, [&] {
                k_meas_det<<<dim3(nb, b.count), DET_WARPS * 32, (size_t)DET_WARPS * det_smem_words(b.H) * 4, s>>>(
                    a, skipped ? l | DET_SKIPPED : l);
            });
            const uint32_t fixed = 4u * (uint32_t)lc.sm_count;
            if (!skipped) launch(kp, STAB_KERNEL_OTHER, s, 0.0, [&] {
                const unsigned long long pairs = (unsigned long long)b.H * b.count;
                k_destab_to_rm<<<(uint32_t)std::min<unsigned long long>(pairs, fixed), 256, 0, s>>>(a);
            });
            cudaError_t er = cudaSuccess;
            if (!skipped) launch(kp, STAB_KERNEL_MEAS_RAND, s, 0.0,
                                 [&] { er = launch_meas_rand(a, l, b.count, lc.rand_cluster, rsm, s); });
            if (er != cudaSuccess) return er;
            if (!skipped) launch(kp, STAB_KERNEL_MEAS_DET, s, 0.0, [&] {
                const unsigned long long ctas = ((unsigned long long)L.count * b.count + DET_WARPS - 1) / DET_WARPS;
                k_meas_late<<<(uint32_t)std::min<unsigned long long>(ctas, 2ull * fixed), DET_WARPS * 32,
                              (size_t)DET_WARPS * 2 * b.H * 4, s>>>(a, l);
            });
            if (L.has_cond) {
                // a following gate run applies the flips as it loads each slice
                if (k + 1 < p.runs.size() && p.runs[k + 1].type == LT_GATE)
                    cond_pending = (int32_t)l;
                else
                    launch(kp, STAB_KERNEL_OTHER, s, 0.0,
                           [&] { k_cond<<<dim3(b.CW, b.count), 256, 0, s>>>(a, l); });
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace stab
