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
//  * k_meas_rand: one CTA per tableau runs the layer's random measurements in
//    circuit order (pivot, rowsum of the pivot into every anticommuting row
//    with the mod-4 phase, destabilizer copy, +-Z_a install; Sec. 2.4), keeping
//    the measured columns of later ops of the layer up to date.
//  * k_cond: the X of resets whose outcome was 1 (and the Z of RESET_ERROR)
//    as sign flips r ^= z_a (x_a); these Paulis commute with the layer's other
//    measurements, so they are applied after it.
#include "device_common.cuh"

#include <algorithm>

namespace stab {

enum : uint8_t { MS_DONE = 0, MS_RANDOM = 1, MS_SKIP = 2 };

struct LArgs {
    DevProg P;
    uint32_t *qm;
    unsigned long long qm_stride;
    uint32_t *rm;
    unsigned long long rm_stride;
    uint32_t RS, Hr;                 // row stride (words) and z offset in a row
    uint32_t *r;
    uint8_t *dirty;
    uint32_t *cols;
    unsigned long long cols_stride;  // words per tableau
    uint8_t *mstat, *mout;
    unsigned long long m_stride;     // items per tableau
    DevStreams st;
    unsigned long long *record;
    unsigned long long rec_stride;
    int *err;
    uint32_t B;
};

static inline uint32_t round4(uint32_t v) { return (v + 3u) & ~3u; }

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
    int32_t cols_layer;
};

__global__ void k_gate_run(LArgs a, GRun g) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t sred[32];
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW;
    const uint32_t w = blockIdx.x, t = blockIdx.y;
    uint32_t *sx = smem, *sz = smem + n;
    uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + (size_t)CW * n;
    uint32_t *rm = a.rm + t * a.rm_stride;
    uint8_t *dirty = a.dirty + (size_t)t * CW;
    const bool dty = dirty[w] != 0;
    if (!dty) {
        for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
            sx[j] = qx[(size_t)w * n + j];
            sz[j] = qz[(size_t)w * n + j];
        }
    } else {
        slice_load_rm(rm, a.RS, a.Hr, H, n, w, [&](uint32_t j, uint32_t x, uint32_t z) {
            sx[j] = x;
            sz[j] = z;
        });
    }
    __syncthreads();
    uint32_t racc = 0;
    for (uint32_t l = g.l0; l < g.l1; l++) {
        const Layer L = a.P.layers[l];
        for (uint32_t i = threadIdx.x; i < L.count; i += blockDim.x) {
            const GItem it = a.P.gitems[L.first + i];
            uint32_t xa = sx[it.a], za = sz[it.a], xb = 0, zb = 0;
            const bool two = it.b != it.a;
            if (two) { xb = sx[it.b]; zb = sz[it.b]; }
            racc ^= apply_item(it, xa, za, xb, zb, a.st, t, a.P.thr);
            sx[it.a] = xa; sz[it.a] = za;
            if (two) { sx[it.b] = xb; sz[it.b] = zb; }
        }
        __syncthreads();
    }
    // sign flips: XOR-reduce over the CTA, one plain update per slice
    for (int o = 16; o; o >>= 1) racc ^= __shfl_xor_sync(FULL_MASK, racc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sred[warp] = racc;
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
        qx[(size_t)w * n + j] = sx[j];
        qz[(size_t)w * n + j] = sz[j];
    }
    if (g.cols_layer >= 0) {
        const Layer M = a.P.layers[g.cols_layer];
        uint32_t *cols = a.cols + t * a.cols_stride;
        for (uint32_t i = threadIdx.x; i < M.count; i += blockDim.x)
            cols[(size_t)i * CW + w] = sx[a.P.mitems[M.first + i].q];
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < nw ? sred[lane] : 0u;
        for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(FULL_MASK, v, o);
        if (lane == 0) {
            a.r[(size_t)t * CW + w] ^= v;
            dirty[w] = 0;
        }
    }
    if (g.want_rm) {
        slice_store_rm(rm, a.RS, a.Hr, H, w,
                       [&](uint32_t j) { return j < n ? sx[j] : 0u; },
                       [&](uint32_t j) { return j < n ? sz[j] : 0u; });
    }
}

// Full column-packed -> row-packed copy (used when a measurement layer comes
// first and the row-packed copy is stale).
__global__ void k_qm_to_rm(LArgs a) {
    const uint32_t n = a.P.n, H = a.P.H, CW = a.P.CW;
    const uint32_t w = blockIdx.x, t = blockIdx.y;
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
__global__ void k_gather_cols(LArgs a, uint32_t layer) {
    const uint32_t n = a.P.n, CW = a.P.CW;
    const uint32_t w = blockIdx.x, t = blockIdx.y;
    const Layer M = a.P.layers[layer];
    const bool dty = a.dirty[(size_t)t * CW + w] != 0;
    const uint32_t *qx = a.qm + t * a.qm_stride;
    const uint32_t *rm = a.rm + t * a.rm_stride;
    uint32_t *cols = a.cols + t * a.cols_stride;
    for (uint32_t i = threadIdx.x; i < M.count; i += blockDim.x) {
        const uint32_t q = a.P.mitems[M.first + i].q;
        cols[(size_t)i * CW + w] = dty ? rm_col_word(rm, a.RS, a.Hr, w, q, false)
                                       : qx[(size_t)w * n + q];
    }
}

// Sign of the product of the stabilizers selected by the destabilizer column
// `colK` (H words), computed by one warp.  For commuting rows P_1..P_k (ascending
// row order) the power of i of the product is
//   2 sum r_b + sum_b popc(x_b & z_b) + 2 sum_{b<b'} popc(z_b & x_b') - popc(X & Z)
// with X = xor of x_b, Z = xor of z_b; the product must be +-Z_q, so X = 0.
// Zp/Xp: per-warp scratch of H words each.
__device__ int det_outcome_warp(const uint32_t *rm, uint32_t RS, uint32_t Hr, uint32_t H,
                                const uint32_t *r, const uint32_t *colK, uint32_t q,
                                uint32_t *Zp, uint32_t *Xp, int *err) {
    const int lane = threadIdx.x & 31;
    for (uint32_t c = lane; c < H; c += 32) { Zp[c] = 0; Xp[c] = 0; }
    __syncwarp();
    int acc = 0, rsum = 0;
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
                const uint32_t s = 32 * H + 32 * u + b;       // stabilizer partner row
                const uint32_t *row = rm + (size_t)s * RS;
                for (uint32_t c = lane; c < H; c += 32) {
                    uint32_t x = row[c], z = row[Hr + c];
                    acc += __popc(x & z) + 2 * __popc(x & Zp[c]);
                    Zp[c] ^= z;
                    Xp[c] ^= x;
                }
                rsum += (int)rbit(r, s);
            }
        }
    }
    bool ok = true;
    for (uint32_t c = lane; c < H; c += 32) {
        uint32_t wantz = (c == (q >> 5)) ? (1u << (q & 31)) : 0u;
        ok &= (Xp[c] == 0u) && (Zp[c] == wantz);
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
    const int e = (acc + 2 * rsum) & 3;
    if (!__all_sync(FULL_MASK, ok)) set_err(err, DERR_BAD_PRODUCT);
    if (e & 1) set_err(err, DERR_ODD_PHASE);
    __syncwarp();
    return (e >> 1) & 1;
}

__device__ __forceinline__ void write_record(const LArgs &a, uint32_t t, uint32_t rec, uint32_t out) {
    if (rec != 0xffffffffu && out)
        atomicOr(&a.record[(unsigned long long)t * a.rec_stride + (rec >> 6)], 1ull << (rec & 63));
}

constexpr int DET_WARPS = 8;

__global__ void __launch_bounds__(DET_WARPS * 32) k_meas_det(LArgs a, uint32_t layer) {
    extern __shared__ uint32_t smem[];
    const uint32_t H = a.P.H, CW = a.P.CW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = blockIdx.y;
    const Layer M = a.P.layers[layer];
    const uint32_t i = blockIdx.x * DET_WARPS + warp;
    if (i >= M.count) return;
    const MItem m = a.P.mitems[M.first + i];
    uint8_t *stat = a.mstat + t * a.m_stride, *out = a.mout + t * a.m_stride;
    if (m.flags & MF_RESET_ERR) {
        const uint32_t u0 = noise_word(a.st, t, m.nl);
        if ((unsigned long long)u0 >= a.P.thr[m.np].t[0]) {
            if (lane == 0) { stat[i] = MS_SKIP; out[i] = 0; }
            return;
        }
    }
    const uint32_t *col = a.cols + t * a.cols_stride + (size_t)i * CW;
    uint32_t nz = 0;
    for (uint32_t c = lane; c < H; c += 32) nz |= col[H + c];
    if (__any_sync(FULL_MASK, nz != 0)) {
        if (lane == 0) stat[i] = MS_RANDOM;
        return;
    }
    uint32_t *Zp = smem + (size_t)warp * 2 * H, *Xp = Zp + H;
    const int o = det_outcome_warp(a.rm + t * a.rm_stride, a.RS, a.Hr, H, a.r + (size_t)t * CW,
                                   col, m.q, Zp, Xp, a.err);
    if (lane == 0) {
        stat[i] = MS_DONE;
        out[i] = (uint8_t)o;
        write_record(a, t, m.rec, (uint32_t)o);
    }
}

// rowsum(s, p) on the row-packed copy by one warp: row s <- row p * row s
// with r_s from 2 r_s + 2 r_p + (power of i) mod 4 (Appendix B).
__device__ __forceinline__ void rowsum_warp(uint32_t *rm, uint32_t RS, uint32_t Hr, uint32_t H,
                                            uint32_t *r, uint32_t s, uint32_t p, int *err) {
    const int lane = threadIdx.x & 31;
    const uint32_t *rp = rm + (size_t)p * RS;
    uint32_t *rs = rm + (size_t)s * RS;
    int acc = 0;
    for (uint32_t c = lane; c < H; c += 32) {
        const uint32_t xp = rp[c], zp = rp[Hr + c], xs = rs[c], zs = rs[Hr + c];
        acc += phase_word(xp, zp, xs, zs);
        rs[c] = xs ^ xp;
        rs[Hr + c] = zs ^ zp;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, o);
    if (lane == 0) {
        const uint32_t r_s = rbit(r, s), r_p = rbit(r, p);
        const int e = (int)(2 * r_s + 2 * r_p) + acc;
        if (e & 1) set_err(err, DERR_ODD_PHASE);
        const uint32_t nr = (uint32_t)((e & 3) >> 1);
        if (nr != r_s) atomicXor(&r[s >> 5], 1u << (s & 31));
    }
}

constexpr int RAND_THREADS = 1024;

__global__ void __launch_bounds__(RAND_THREADS) k_meas_rand(LArgs a, uint32_t layer) {
    extern __shared__ uint32_t smem[];      // 2H words for the det fallback
    __shared__ int s_pw;
    const uint32_t H = a.P.H, CW = a.P.CW, RS = a.RS, Hr = a.Hr;
    const uint32_t t = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const Layer M = a.P.layers[layer];
    uint8_t *stat = a.mstat + t * a.m_stride, *out = a.mout + t * a.m_stride;
    uint32_t *cols = a.cols + t * a.cols_stride;
    uint32_t *rm = a.rm + t * a.rm_stride;
    uint32_t *r = a.r + (size_t)t * CW;
    uint8_t *dirty = a.dirty + (size_t)t * CW;
    for (uint32_t i = 0; i < M.count; i++) {
        if (stat[i] != MS_RANDOM) continue;          // block-uniform (written by earlier kernels / step)
        const MItem m = a.P.mitems[M.first + i];
        const uint32_t *col = cols + (size_t)i * CW;
        if (threadIdx.x == 0) s_pw = 0x7fffffff;
        __syncthreads();
        for (uint32_t c = threadIdx.x; c < H; c += blockDim.x)
            if (col[H + c]) atomicMin(&s_pw, (int)c);
        __syncthreads();
        const int pw = s_pw;
        if (pw == 0x7fffffff) {
            // became deterministic after an earlier random measurement of this layer
            if (warp == 0) {
                const int o = det_outcome_warp(rm, RS, Hr, H, r, col, m.q, smem, smem + H, a.err);
                if (lane == 0) {
                    out[i] = (uint8_t)o;
                    stat[i] = MS_DONE;
                    write_record(a, t, m.rec, (uint32_t)o);
                }
            }
            __syncthreads();
            continue;
        }
        const uint32_t pword = col[H + pw];
        const uint32_t q = 32u * (uint32_t)pw + (uint32_t)(__ffs(pword) - 1);  // destabilizer slot
        const uint32_t p = 32u * H + q;                                          // pivot (stabilizer) slot
        const uint32_t coin = (m.flags & MF_RESET_ERR) ? (noise_word(a.st, t, m.nl + 1) & 1u)
                                                       : coin_bit(a.st, t, m.coin);
        // rowsum(s, p) for every row s != p with x_{s,a} = 1.  Row q (= p - n)
        // is skipped: it is overwritten by row p below, and its product with p
        // has an odd power of i, which Appendix B leaves the sign bit unchanged for.
        for (uint32_t w = (uint32_t)warp; w < CW; w += (uint32_t)nw) {
            uint32_t mask = col[w];
            if (lane == 0 && mask) dirty[w] = 1;
            if (w == (p >> 5)) mask &= ~(1u << (p & 31));
            if (w == (q >> 5)) mask &= ~(1u << (q & 31));
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                rowsum_warp(rm, RS, Hr, H, r, 32 * w + b, p, a.err);
            }
        }
        __syncthreads();
        // row q <- row p; row p <- +-Z_a with sign = coin
        for (uint32_t c = threadIdx.x; c < H; c += blockDim.x) {
            const uint32_t xv = rm[(size_t)p * RS + c], zv = rm[(size_t)p * RS + Hr + c];
            rm[(size_t)q * RS + c] = xv;
            rm[(size_t)q * RS + Hr + c] = zv;
            rm[(size_t)p * RS + c] = 0u;
            rm[(size_t)p * RS + Hr + c] = (c == (m.q >> 5)) ? (1u << (m.q & 31)) : 0u;
        }
        if (threadIdx.x == 0) {
            const uint32_t rp = rbit(r, p);
            r[q >> 5] = (r[q >> 5] & ~(1u << (q & 31))) | (rp << (q & 31));
            r[p >> 5] = (r[p >> 5] & ~(1u << (p & 31))) | (coin << (p & 31));
            dirty[p >> 5] = 1;
            dirty[q >> 5] = 1;
        }
        // keep the measured columns of later random ops current:
        // rows in A get x ^= x_{p,b}; row q gets x_{p,b}; row p gets 0.
        for (uint32_t j = i + 1 + (uint32_t)warp; j < M.count; j += (uint32_t)nw) {
            if (stat[j] != MS_RANDOM) continue;
            uint32_t *cj = cols + (size_t)j * CW;
            const uint32_t bp = (cj[p >> 5] >> (p & 31)) & 1u;
            if (bp) {
                for (uint32_t c = lane; c < CW; c += 32) {
                    uint32_t v = col[c];
                    if (c == (p >> 5)) v &= ~(1u << (p & 31));
                    cj[c] ^= v;
                }
            }
            __syncwarp();
            if (lane == 0) {
                cj[q >> 5] = (cj[q >> 5] & ~(1u << (q & 31))) | (bp << (q & 31));
                cj[p >> 5] &= ~(1u << (p & 31));
            }
            __syncwarp();
        }
        if (threadIdx.x == 0) {
            out[i] = (uint8_t)coin;
            stat[i] = MS_DONE;
            write_record(a, t, m.rec, coin);
        }
        __syncthreads();
    }
}

// X after resets with outcome 1 (r ^= z_a) and RESET_ERROR's Z (r ^= x_a).
__global__ void k_cond(LArgs a, uint32_t layer) {
    __shared__ uint32_t sred[32];
    const uint32_t n = a.P.n, CW = a.P.CW;
    const uint32_t w = blockIdx.x, t = blockIdx.y;
    const Layer M = a.P.layers[layer];
    const bool dty = a.dirty[(size_t)t * CW + w] != 0;
    const uint32_t *qx = a.qm + t * a.qm_stride, *qz = qx + (size_t)CW * n;
    const uint32_t *rm = a.rm + t * a.rm_stride;
    const uint8_t *stat = a.mstat + t * a.m_stride, *out = a.mout + t * a.m_stride;
    uint32_t v = 0;
    for (uint32_t i = threadIdx.x; i < M.count; i += blockDim.x) {
        const MItem m = a.P.mitems[M.first + i];
        if (!m.flags) continue;
        bool fx = false, fz = false;
        if (m.flags & MF_RESET) fx = out[i] != 0;
        if (m.flags & MF_RESET_ERR) {
            fx = stat[i] == MS_DONE && out[i] != 0;
            const uint32_t u2 = noise_word(a.st, t, m.nl + 2);
            fz = (unsigned long long)u2 < a.P.thr[m.np].t[1];
        }
        if (fx) v ^= dty ? rm_col_word(rm, a.RS, a.Hr, w, m.q, true) : qz[(size_t)w * n + m.q];
        if (fz) v ^= dty ? rm_col_word(rm, a.RS, a.Hr, w, m.q, false) : qx[(size_t)w * n + m.q];
    }
    for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(FULL_MASK, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t u = lane < nw ? sred[lane] : 0u;
        for (int o = 16; o; o >>= 1) u ^= __shfl_xor_sync(FULL_MASK, u, o);
        if (lane == 0 && u) a.r[(size_t)t * CW + w] ^= u;
    }
}

// ---------------------------------------------------------------- host side
size_t layered_gate_smem(uint32_t n) { return (size_t)8 * n; }

int layered_supported(uint32_t n, const LaunchCfg &lc) {
    return layered_gate_smem(n) + 1024 <= lc.smem_optin;
}

size_t batch_bytes(uint32_t n, uint32_t count) {
    const size_t H = (n + 31) / 32, CW = 2 * H, Hr = round4((uint32_t)H), RS = 2 * Hr;
    size_t per = 4 * (2 * CW * (size_t)n + 64 * H * RS + CW) + CW;
    return per * count + 1024;
}

int batch_alloc(Batch &b, uint32_t n, uint32_t count, std::string *err) {
    batch_free(b);
    b.n = n;
    b.H = (n + 31) / 32;
    b.CW = 2 * b.H;
    b.count = count;
    const size_t Hr = round4(b.H), RS = 2 * Hr;
    b.qm_stride = 2 * (size_t)b.CW * n;
    b.rm_stride = 64 * (size_t)b.H * RS;
    const size_t qm_b = 4 * b.qm_stride * count, rm_b = 4 * b.rm_stride * count;
    const size_t r_b = 4 * (size_t)b.CW * count, d_b = (size_t)b.CW * count;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    b.bytes = up(qm_b) + up(rm_b) + up(r_b) + up(d_b);
    if (cudaMalloc(&b.mem, b.bytes) != cudaSuccess) {
        cudaGetLastError();
        b.mem = nullptr;
        *err = "cudaMalloc of " + std::to_string(b.bytes) + " bytes for tableaux failed";
        return STAB_ERR_OOM;
    }
    char *p = (char *)b.mem;
    b.qm = (uint32_t *)p; p += up(qm_b);
    b.rm = (uint32_t *)p; p += up(rm_b);
    b.r = (uint32_t *)p; p += up(r_b);
    b.dirty = (uint8_t *)p;
    b.rm_valid = false;
    return STAB_OK;
}

void batch_free(Batch &b) {
    if (b.mem) cudaFree(b.mem);
    b = Batch{};
}

static LArgs make_args(const HostProg *p, Batch &b, MeasScratch *ms, const DevStreams *st,
                       unsigned long long *record, size_t rec_stride, int *d_err) {
    LArgs a{};
    if (p) a.P = p->dev;
    a.P.n = b.n; a.P.H = b.H; a.P.CW = b.CW;
    a.qm = b.qm; a.qm_stride = b.qm_stride;
    a.rm = b.rm; a.rm_stride = b.rm_stride;
    a.Hr = round4(b.H); a.RS = 2 * a.Hr;
    a.r = b.r; a.dirty = b.dirty;
    if (ms && p) {
        a.cols = ms->cols;
        a.cols_stride = (unsigned long long)std::max<uint32_t>(1, p->dev.max_meas) * b.CW;
        a.mstat = ms->stat; a.mout = ms->out;
        a.m_stride = std::max<uint32_t>(1, p->dev.max_meas);
    }
    if (st) a.st = *st;
    a.record = record;
    a.rec_stride = rec_stride;
    a.err = d_err;
    a.B = b.count;
    return a;
}

cudaError_t layered_init(Batch &b, cudaStream_t s) {
    LArgs a = make_args(nullptr, b, nullptr, nullptr, nullptr, 0, nullptr);
    k_init<<<1024, 256, 0, s>>>(a);
    b.rm_valid = true;
    return cudaGetLastError();
}

cudaError_t layered_sync_qm(Batch &b, cudaStream_t s) {
    LArgs a = make_args(nullptr, b, nullptr, nullptr, nullptr, 0, nullptr);
    k_rm_to_qm<<<dim3(b.CW, b.count), 256, 0, s>>>(a);
    return cudaGetLastError();
}

static bool g_attr_set = false;

cudaError_t layered_run(const HostProg &p, Batch &b, MeasScratch &ms, const DevStreams &st,
                        unsigned long long *record, size_t rec_stride, int *d_err,
                        const LaunchCfg &lc, cudaStream_t s) {
    if (!g_attr_set) {
        cudaFuncSetAttribute(k_gate_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(lc.smem_optin - 1024));
        cudaFuncSetAttribute(k_meas_det, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(lc.smem_optin - 1024));
        cudaFuncSetAttribute(k_meas_rand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(lc.smem_optin - 1024));
        g_attr_set = true;
    }
    LArgs a = make_args(&p, b, &ms, &st, record, rec_stride, d_err);
    const uint32_t gthreads = std::min<uint32_t>(512, std::max<uint32_t>(64, (p.dev.max_gitems + 31) / 32 * 32));
    const size_t gsm = layered_gate_smem(b.n);
    bool cols_ready = false;
    for (size_t k = 0; k < p.runs.size(); k++) {
        const Run &R = p.runs[k];
        if (R.type == LT_GATE) {
            GRun g{};
            g.l0 = R.l0; g.l1 = R.l1;
            const bool next_meas = k + 1 < p.runs.size() && p.runs[k + 1].type == LT_MEAS;
            g.want_rm = next_meas ? 1u : 0u;
            g.cols_layer = next_meas ? (int32_t)p.runs[k + 1].l0 : -1;
            k_gate_run<<<dim3(b.CW, b.count), gthreads, gsm, s>>>(a, g);
            b.rm_valid = next_meas;
            cols_ready = next_meas;
        } else {
            const uint32_t l = R.l0;
            const Layer &L = p.layers[l];
            if (!b.rm_valid) {
                k_qm_to_rm<<<dim3(b.CW, b.count), 256, 0, s>>>(a);
                b.rm_valid = true;
            }
            if (!cols_ready)
                k_gather_cols<<<dim3(b.CW, b.count), 256, 0, s>>>(a, l);
            const uint32_t nb = (L.count + DET_WARPS - 1) / DET_WARPS;
            k_meas_det<<<dim3(nb, b.count), DET_WARPS * 32, (size_t)DET_WARPS * 2 * b.H * 4, s>>>(a, l);
            k_meas_rand<<<b.count, RAND_THREADS, (size_t)2 * b.H * 4, s>>>(a, l);
            if (L.has_cond)
                k_cond<<<dim3(b.CW, b.count), 256, 0, s>>>(a, l);
            cols_ready = false;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace stab
