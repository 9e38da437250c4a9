// resident.cu -- the resident engine: each tableau lives in shared memory for
// its whole circuit; a persistent launch runs many shots of many circuits
// (uneven qubit counts) at once.  A CTA holds `tableaux_per_cta` groups of
// `group_threads` threads; each group pulls shots from a device work counter,
// simulates the shot from |0...0> to its last op, writes its record and pulls
// the next one.  Synchronisation is group-local (warp sync or a named barrier).
//
// Per shot the circuit is the same CHP evolution as the layered engine
// (Sec. 2.4 gate table, Appendix B rowsum, Sec. 2.4 measurement rules), here on
// a column-packed tableau in shared memory: x[j][w], z[j][w] hold rows
// 32w..32w+31 of column j, so a gate touches CW contiguous words per column.
#include "device_common.cuh"
#include "ctx.h"

#include <algorithm>
#include <cstring>

namespace stab {

struct GroupCtx {
    uint32_t gtid, G, gid;
};

__device__ __forceinline__ void gsync(const GroupCtx &g) {
    if (g.G == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(g.gid + 1), "r"(g.G) : "memory");
}

// smem layout per group (32-bit words): x[n*CW], z[n*CW], r[CW], cnt[64H] (int),
// acol[CW] (snapshot of the measured column), prow[n] (pivot row Pauli per
// column), mflag[n] bytes (per-op class within a measurement layer), misc[8]
__host__ __device__ __forceinline__ size_t res_words(uint32_t n) {
    const size_t H = (n + 31) / 32, CW = 2 * H;
    return 2 * (size_t)n * CW + CW + 64 * H + CW + n + (n + 3) / 4 + 8;
}

// Deterministic outcome of measuring Z_a by one warp of the group: sign of the
// product of the stabilizers selected by the destabilizer half of column a
// (ordered-product closed form, evaluated column by column).
__device__ uint32_t res_det_warp(uint32_t n, uint32_t H, uint32_t CW, const uint32_t *X, const uint32_t *Z,
                                 const uint32_t *r, uint32_t a, int *err) {
    const int lane = threadIdx.x & 31;
    const uint32_t *K = X + (size_t)a * CW;
    int acc = 0;
    uint32_t bad = 0;
    for (uint32_t j = lane; j < n; j += 32) {
        const uint32_t *xj = X + (size_t)j * CW + H, *zj = Z + (size_t)j * CW + H;
        uint32_t carry = 0, px = 0, pz = 0;
        for (uint32_t w = 0; w < H; w++) {
            const uint32_t k = K[w];
            if (!k) continue;
            const uint32_t kx = xj[w] & k, kz = zj[w] & k;
            uint32_t pre = kz;
            pre ^= pre << 1; pre ^= pre << 2; pre ^= pre << 4; pre ^= pre << 8; pre ^= pre << 16;
            pre <<= 1;
            acc += __popc(kx & kz) + 2 * ((__popc(kx & pre) + (int)(carry & __popc(kx))) & 1);
            carry ^= __popc(kz) & 1u;
            px ^= __popc(kx) & 1u;
            pz ^= __popc(kz) & 1u;
        }
        bad |= px | (pz ^ (j == a ? 1u : 0u));
    }
    for (uint32_t w = lane; w < H; w += 32) acc += 2 * __popc(r[H + w] & K[w]);
    acc = __reduce_add_sync(FULL_MASK, acc);
    bad = __reduce_or_sync(FULL_MASK, bad);
    if (lane == 0) {
        if (acc & 1) set_err(err, DERR_ODD_PHASE);
        if (bad) set_err(err, DERR_BAD_PRODUCT);
    }
    return (uint32_t)(acc >> 1) & 1u;
}

size_t resident_smem_per_tableau(uint32_t n) { return 4 * res_words(n); }

int resident_supported(uint32_t n, const LaunchCfg &lc) {
    return resident_smem_per_tableau(n) + 64 <= lc.smem_optin;
}

// rowsum(s, p) for every row s set in the snapshot `acol` except the pivot
// p and its destabilizer partner q (Appendix B, column by column): x/z update
// and per-row power of i, then the signs.  prow[j] & 3 = the pivot row's
// Pauli in column j (1 x, 2 z).  Returns the pivot row's sign.
__device__ uint32_t res_rowsum_rows(const GroupCtx &g, uint32_t n, uint32_t CW, uint32_t *X, uint32_t *Z,
                                    uint32_t *r, int *cnt, const uint32_t *acol, const uint32_t *prow,
                                    uint32_t pwd, uint32_t qwd, uint32_t pm, uint32_t qm, int *err) {
    const uint32_t *colA = acol;
    for (uint32_t idx = g.gtid; idx < n * CW; idx += g.G) {
        const uint32_t j = idx / CW, w = idx - j * CW;
        const uint32_t P = prow[j] & 3u;
        if (!P) continue;
        uint32_t M = colA[w];
        if (w == pwd) M &= ~pm;
        if (w == qwd) M &= ~qm;
        if (!M) continue;
        uint32_t &xw = X[(size_t)j * CW + w], &zw = Z[(size_t)j * CW + w];
        const uint32_t x = xw, z = zw;
        uint32_t plus, minus;
        if (P == 1) { plus = z & x; minus = z & ~x; }          // pivot X: g = z(2x-1)
        else if (P == 3) { plus = z & ~x; minus = x & ~z; }    // pivot Y: g = z - x
        else { plus = x & ~z; minus = x & z; }                 // pivot Z: g = x(1-2z)
        plus &= M; minus &= M;
        if (P & 1u) xw = x ^ M;
        if (P & 2u) zw = z ^ M;
        while (plus) { const int b = __ffs(plus) - 1; plus &= plus - 1; atomicAdd(&cnt[32 * w + b], 1); }
        while (minus) { const int b = __ffs(minus) - 1; minus &= minus - 1; atomicAdd(&cnt[32 * w + b], -1); }
    }
    gsync(g);
    const uint32_t rp = (r[pwd] & pm) ? 1u : 0u;
    for (uint32_t w = g.gtid; w < CW; w += g.G) {
        uint32_t M = colA[w];
        if (w == pwd) M &= ~pm;
        if (w == qwd) M &= ~qm;
        uint32_t flip = 0;
        while (M) {
            const int b = __ffs(M) - 1;
            M &= M - 1;
            const uint32_t rs = (r[w] >> b) & 1u;
            const int e = (int)(2 * rs + 2 * rp) + cnt[32 * w + b];
            if (e & 1) set_err(err, DERR_ODD_PHASE);
            if ((uint32_t)((e & 3) >> 1) != rs) flip |= 1u << b;
        }
        if (flip) r[w] ^= flip;          // each word owned by one thread here
    }
    gsync(g);
    return rp;
}

// Z measurement of qubit a in the group's shared-memory tableau.
// Returns the outcome; `coin` is used only if the outcome is random.
__device__ uint32_t res_measure(const GroupCtx &g, uint32_t n, uint32_t H, uint32_t CW,
                                uint32_t *X, uint32_t *Z, uint32_t *r, int *cnt, uint32_t *acol,
                                uint32_t *prow, uint32_t *misc, uint32_t a, uint32_t coin, int *err) {
    // ---- pivot search: first stabilizer word of column a with a set bit
    if (g.gtid == 0) misc[0] = 0x7fffffffu;
    gsync(g);
    for (uint32_t w = g.gtid; w < H; w += g.G)
        if (X[(size_t)a * CW + H + w]) atomicMin(&misc[0], w);
    gsync(g);
    const uint32_t pw = misc[0];
    if (pw == 0x7fffffffu) {
        // ---- deterministic: sign of prod of stabilizers selected by the
        // destabilizer half of column a (ordered-product closed form)
        if (g.gtid == 0) { misc[1] = 0; misc[2] = 0; }
        gsync(g);
        int acc = 0;
        uint32_t bad = 0;
        const uint32_t *K = X + (size_t)a * CW;         // destabilizer words [0, H)
        for (uint32_t j = g.gtid; j < n; j += g.G) {
            const uint32_t *xj = X + (size_t)j * CW + H, *zj = Z + (size_t)j * CW + H;
            uint32_t carry = 0, px = 0, pz = 0;
            for (uint32_t w = 0; w < H; w++) {
                const uint32_t k = K[w];
                if (!k) continue;
                const uint32_t kx = xj[w] & k, kz = zj[w] & k;
                uint32_t pre = kz;
                pre ^= pre << 1; pre ^= pre << 2; pre ^= pre << 4; pre ^= pre << 8; pre ^= pre << 16;
                pre <<= 1;                                 // exclusive prefix xor
                acc += __popc(kx & kz) + 2 * ((__popc(kx & pre) + (int)(carry & __popc(kx))) & 1);
                carry ^= __popc(kz) & 1u;
                px ^= __popc(kx) & 1u;
                pz ^= __popc(kz) & 1u;
            }
            bad |= px | (pz ^ (j == a ? 1u : 0u));
        }
        for (uint32_t w = g.gtid; w < H; w += g.G) acc += 2 * __popc(r[H + w] & K[w]);
        acc = __reduce_add_sync(FULL_MASK, acc);
        bad = __reduce_or_sync(FULL_MASK, bad);
        if ((g.gtid & 31) == 0) {
            atomicAdd(&misc[1], (uint32_t)acc);
            if (bad) misc[2] = 1;
        }
        gsync(g);
        const uint32_t e = misc[1] & 3u;
        if (g.gtid == 0) {
            if (e & 1u) set_err(err, DERR_ODD_PHASE);
            if (misc[2]) set_err(err, DERR_BAD_PRODUCT);
        }
        gsync(g);
        return (e >> 1) & 1u;
    }
    // ---- random
    const uint32_t pbit = __ffs(X[(size_t)a * CW + H + pw]) - 1;
    const uint32_t q = 32 * pw + pbit, p = 32 * H + q;
    const uint32_t pwd = p >> 5, qwd = q >> 5;
    const uint32_t pm = 1u << (p & 31), qm = 1u << (q & 31);
    // pivot row Pauli per column (2 bits), snapshot of column a (the rowsum
    // below rewrites it), zero the row counters
    for (uint32_t w = g.gtid; w < CW; w += g.G) acol[w] = X[(size_t)a * CW + w];
    for (uint32_t j = g.gtid; j < n; j += g.G)
        prow[j] = ((X[(size_t)j * CW + pwd] & pm) ? 1u : 0u) | ((Z[(size_t)j * CW + pwd] & pm) ? 2u : 0u);
    for (uint32_t s = g.gtid; s < 64 * H; s += g.G) cnt[s] = 0;
    gsync(g);
    const uint32_t rp = res_rowsum_rows(g, n, CW, X, Z, r, cnt, acol, prow, pwd, qwd, pm, qm, err);
    // row q <- row p, row p <- +-Z_a (column by column; bits p and q of a
    // column are handled by one thread)
    for (uint32_t j = g.gtid; j < n; j += g.G) {
        const uint32_t P = prow[j];
        uint32_t *xq = X + (size_t)j * CW + qwd, *zq = Z + (size_t)j * CW + qwd;
        *xq = (P & 1u) ? (*xq | qm) : (*xq & ~qm);
        *zq = (P & 2u) ? (*zq | qm) : (*zq & ~qm);
        X[(size_t)j * CW + pwd] &= ~pm;
        if (j == a) Z[(size_t)j * CW + pwd] |= pm;
        else Z[(size_t)j * CW + pwd] &= ~pm;
    }
    if (g.gtid == 0) {
        r[qwd] = rp ? (r[qwd] | qm) : (r[qwd] & ~qm);
        r[pwd] = coin ? (r[pwd] | pm) : (r[pwd] & ~pm);
    }
    gsync(g);
    return coin;
}

// Measurement of the Pauli product P of `nf` packed factors (qubit | code << 30,
// code 1 X, 2 Y, 3 Z) in the group's tableau.  A row anticommutes with P iff
// x_P . z_S + z_P . x_S is odd (Sec. 3.2), so the column of anticommuting rows
// is the XOR of the factor columns (z for X/Y factors, x for Y/Z factors);
// the rest is the Z measurement with that column in place of x_a, and P in
// place of Z_a as the new stabilizer row.  Returns the outcome.
__device__ uint32_t res_measure_mpp(const GroupCtx &g, uint32_t n, uint32_t H, uint32_t CW,
                                    uint32_t *X, uint32_t *Z, uint32_t *r, int *cnt, uint32_t *acol,
                                    uint32_t *prow, uint32_t *misc, const uint32_t *fac, uint32_t nf,
                                    uint32_t coin, int *err) {
    // P per column in prow bits 2..3 (4 = x, 8 = z)
    for (uint32_t j = g.gtid; j < n; j += g.G) prow[j] = 0;
    gsync(g);
    for (uint32_t i = g.gtid; i < nf; i += g.G) {
        const uint32_t f = fac[i], c = f >> 30;
        prow[f & 0x3fffffffu] = (c <= 2 ? 4u : 0u) | (c >= 2 ? 8u : 0u);
    }
    for (uint32_t w = g.gtid; w < CW; w += g.G) {
        uint32_t v = 0;
        for (uint32_t i = 0; i < nf; i++) {
            const uint32_t f = fac[i], c = f >> 30, q = f & 0x3fffffffu;
            if (c <= 2) v ^= Z[(size_t)q * CW + w];
            if (c >= 2) v ^= X[(size_t)q * CW + w];
        }
        acol[w] = v;
    }
    if (g.gtid == 0) misc[0] = 0x7fffffffu;
    gsync(g);
    for (uint32_t w = g.gtid; w < H; w += g.G)
        if (acol[H + w]) atomicMin(&misc[0], w);
    gsync(g);
    const uint32_t pw = misc[0];
    if (pw == 0x7fffffffu) {
        // deterministic: P = +-(product of the stabilizers whose destabilizers
        // anticommute with P); sign by the ordered-product closed form, whose
        // last term removes the i per Y of the product
        if (g.gtid == 0) { misc[1] = 0; misc[2] = 0; }
        gsync(g);
        int acc = 0;
        uint32_t bad = 0;
        const uint32_t *K = acol;
        for (uint32_t j = g.gtid; j < n; j += g.G) {
            const uint32_t *xj = X + (size_t)j * CW + H, *zj = Z + (size_t)j * CW + H;
            uint32_t carry = 0, px = 0, pz = 0;
            for (uint32_t w = 0; w < H; w++) {
                const uint32_t k = K[w];
                if (!k) continue;
                const uint32_t kx = xj[w] & k, kz = zj[w] & k;
                uint32_t pre = kz;
                pre ^= pre << 1; pre ^= pre << 2; pre ^= pre << 4; pre ^= pre << 8; pre ^= pre << 16;
                pre <<= 1;
                acc += __popc(kx & kz) + 2 * ((__popc(kx & pre) + (int)(carry & __popc(kx))) & 1);
                carry ^= __popc(kz) & 1u;
                px ^= __popc(kx) & 1u;
                pz ^= __popc(kz) & 1u;
            }
            const uint32_t want = prow[j] >> 2;
            bad |= (px ^ (want & 1u)) | (pz ^ (want >> 1));
            acc -= (int)(px & pz);
        }
        for (uint32_t w = g.gtid; w < H; w += g.G) acc += 2 * __popc(r[H + w] & K[w]);
        acc = __reduce_add_sync(FULL_MASK, acc);
        bad = __reduce_or_sync(FULL_MASK, bad);
        if ((g.gtid & 31) == 0) {
            atomicAdd(&misc[1], (uint32_t)acc);
            if (bad) misc[2] = 1;
        }
        gsync(g);
        const uint32_t e = misc[1] & 3u;
        if (g.gtid == 0) {
            if (e & 1u) set_err(err, DERR_ODD_PHASE);
            if (misc[2]) set_err(err, DERR_BAD_PRODUCT);
        }
        gsync(g);
        return (e >> 1) & 1u;
    }
    // random: pivot p = first stabilizer anticommuting with P
    const uint32_t pbit = __ffs(acol[H + pw]) - 1;
    const uint32_t q = 32 * pw + pbit, p = 32 * H + q;
    const uint32_t pwd = p >> 5, qwd = q >> 5;
    const uint32_t pm = 1u << (p & 31), qm = 1u << (q & 31);
    for (uint32_t j = g.gtid; j < n; j += g.G)
        prow[j] |= ((X[(size_t)j * CW + pwd] & pm) ? 1u : 0u) | ((Z[(size_t)j * CW + pwd] & pm) ? 2u : 0u);
    for (uint32_t s = g.gtid; s < 64 * H; s += g.G) cnt[s] = 0;
    gsync(g);
    const uint32_t rp = res_rowsum_rows(g, n, CW, X, Z, r, cnt, acol, prow, pwd, qwd, pm, qm, err);
    // row q <- row p, row p <- (-1)^coin P
    for (uint32_t j = g.gtid; j < n; j += g.G) {
        const uint32_t Pv = prow[j];
        uint32_t *xq = X + (size_t)j * CW + qwd, *zq = Z + (size_t)j * CW + qwd;
        *xq = (Pv & 1u) ? (*xq | qm) : (*xq & ~qm);
        *zq = (Pv & 2u) ? (*zq | qm) : (*zq & ~qm);
        uint32_t *xp = X + (size_t)j * CW + pwd, *zp = Z + (size_t)j * CW + pwd;
        *xp = (Pv & 4u) ? (*xp | pm) : (*xp & ~pm);
        *zp = (Pv & 8u) ? (*zp | pm) : (*zp & ~pm);
    }
    if (g.gtid == 0) {
        r[qwd] = rp ? (r[qwd] | qm) : (r[qwd] & ~qm);
        r[pwd] = coin ? (r[pwd] | pm) : (r[pwd] & ~pm);
    }
    gsync(g);
    return coin;
}

template <int WPT>
__global__ void k_resident(const ResJob *__restrict__ jobs, uint32_t n_jobs, unsigned int *counter,
                           int *err, uint32_t G, uint32_t group_words) {
    extern __shared__ uint32_t smem[];
    GroupCtx g;
    g.G = G;
    g.gid = threadIdx.x / G;
    g.gtid = threadIdx.x - g.gid * G;
    uint32_t *base = smem + (size_t)g.gid * group_words;
    for (;;) {
        if (g.gtid == 0) base[group_words - 1] = atomicAdd(counter, 1u);
        gsync(g);
        const uint32_t jid = base[group_words - 1];
        gsync(g);
        if (jid >= n_jobs) break;
        const ResJob job = jobs[jid];
        const DevProg P = *job.prog;
        const uint32_t n = P.n, H = P.H, CW = P.CW;
        uint32_t *X = base, *Z = X + (size_t)n * CW, *r = Z + (size_t)n * CW;
        int *cnt = (int *)(r + CW);
        uint32_t *acol = (uint32_t *)(cnt + 64 * H), *prow = acol + CW, *misc = prow + n + (n + 3) / 4;
        // |0...0>: destabilizer i = X_i (slot i), stabilizer i = Z_i (slot 32H+i)
        for (uint32_t e = g.gtid; e < n * CW; e += G) {
            const uint32_t j = e / CW, w = e - j * CW;
            X[e] = (w == (j >> 5)) ? (1u << (j & 31)) : 0u;
            Z[e] = (w == H + (j >> 5)) ? (1u << (j & 31)) : 0u;
        }
        for (uint32_t w = g.gtid; w < CW; w += G) r[w] = 0;
        gsync(g);
        const uint32_t nch = (CW + WPT - 1) / WPT;
        for (uint32_t l = 0; l < P.n_layers; l++) {
            const Layer L = P.layers[l];
            if (L.type == LT_GATE) {
                const uint32_t total = L.count * nch;
                for (uint32_t idx = g.gtid; idx < total; idx += G) {
                    const uint32_t it_i = idx / nch, ch = idx - it_i * nch;
                    const GItem it = P.gitems[L.first + it_i];
                    const bool two = it.b != it.a;
#pragma unroll
                    for (int k = 0; k < WPT; k++) {
                        const uint32_t w = ch * WPT + k;
                        if (w >= CW) break;
                        uint32_t xa = X[(size_t)it.a * CW + w], za = Z[(size_t)it.a * CW + w];
                        uint32_t xb = 0, zb = 0;
                        if (two) { xb = X[(size_t)it.b * CW + w]; zb = Z[(size_t)it.b * CW + w]; }
                        const uint32_t rr = apply_item(it, xa, za, xb, zb, job.st, job.shot, P.thr);
                        X[(size_t)it.a * CW + w] = xa; Z[(size_t)it.a * CW + w] = za;
                        if (two) { X[(size_t)it.b * CW + w] = xb; Z[(size_t)it.b * CW + w] = zb; }
                        if (rr) atomicXor(&r[w], rr);
                    }
                }
                gsync(g);
            } else {
                // measurement layer: deterministic outcomes do not depend on the
                // layer's other Z measurements, so they are resolved first, in
                // parallel from the layer's starting state (one warp per op);
                // the random ones then run in circuit order.
                uint8_t *mflag = (uint8_t *)(prow + n);
                const uint32_t gw = g.gtid >> 5, ngw = G >> 5;
                for (uint32_t i = gw; i < L.count; i += ngw) {
                    const MItem m = P.mitems[L.first + i];
                    uint32_t any = 0;
                    if (!(m.flags & (MF_RESET_ERR | MF_MPP)))
                        for (uint32_t w = g.gtid & 31; w < H; w += 32) any |= X[(size_t)m.q * CW + H + w];
                    any = __any_sync(FULL_MASK, any != 0);
                    // Pauli products run in order with the random ones (res_measure_mpp decides)
                    if ((g.gtid & 31) == 0)
                        mflag[i] = (m.flags & MF_RESET_ERR) ? 2 : ((any || (m.flags & MF_MPP)) ? 1 : 0);
                }
                gsync(g);
                for (uint32_t i = gw; i < L.count; i += ngw) {
                    if (mflag[i] != 0) continue;
                    const MItem m = P.mitems[L.first + i];
                    const uint32_t o = res_det_warp(n, H, CW, X, Z, r, m.q, err);
                    if ((g.gtid & 31) == 0) {
                        if (m.rec != 0xffffffffu && o)
                            atomicOr(&job.record[(unsigned long long)job.shot * job.rec_stride + (m.rec >> 6)],
                                     1ull << (m.rec & 63));
                        if (o && (m.flags & (MF_RESET | MF_RESET_AFTER))) mflag[i] = 3;
                    }
                }
                gsync(g);
                // X after deterministic resets whose outcome was 1 (commutes with
                // the layer's other measurements)
                for (uint32_t i = 0; i < L.count; i++) {
                    if (mflag[i] != 3) continue;          // group-uniform
                    const uint32_t q = P.mitems[L.first + i].q;
                    for (uint32_t w = g.gtid; w < CW; w += G) r[w] ^= Z[(size_t)q * CW + w];
                }
                gsync(g);
                for (uint32_t i = 0; i < L.count; i++) {
                    if (mflag[i] != 1 && mflag[i] != 2) continue;
                    const MItem m = P.mitems[L.first + i];
                    uint32_t coin;
                    if (m.flags & MF_RESET_ERR) {
                        const uint32_t u0 = noise_word(job.st, job.shot, m.nl);
                        if ((unsigned long long)u0 < P.thr[m.np].t[0]) {
                            coin = noise_word(job.st, job.shot, m.nl + 1) & 1u;
                            const uint32_t o = res_measure(g, n, H, CW, X, Z, r, cnt, acol, prow, misc, m.q, coin, err);
                            if (o) for (uint32_t w = g.gtid; w < CW; w += G) r[w] ^= Z[(size_t)m.q * CW + w];
                            gsync(g);
                        }
                        const uint32_t u2 = noise_word(job.st, job.shot, m.nl + 2);
                        if ((unsigned long long)u2 < P.thr[m.np].t[1]) {
                            for (uint32_t w = g.gtid; w < CW; w += G) r[w] ^= X[(size_t)m.q * CW + w];
                            gsync(g);
                        }
                        continue;
                    }
                    coin = coin_bit(job.st, job.shot, m.coin);
                    const uint32_t o = (m.flags & MF_MPP)
                        ? res_measure_mpp(g, n, H, CW, X, Z, r, cnt, acol, prow, misc, P.mfactors + m.nl, m.np, coin, err)
                        : res_measure(g, n, H, CW, X, Z, r, cnt, acol, prow, misc, m.q, coin, err);
                    if (m.rec != 0xffffffffu && o && g.gtid == 0)
                        atomicOr(&job.record[(unsigned long long)job.shot * job.rec_stride + (m.rec >> 6)],
                                 1ull << (m.rec & 63));
                    if (o && (m.flags & (MF_RESET | MF_RESET_AFTER))) {   // X_a flips rows with z_a = 1
                        for (uint32_t w = g.gtid; w < CW; w += G) r[w] ^= Z[(size_t)m.q * CW + w];
                        gsync(g);
                    }
                }
            }
        }
        gsync(g);
    }
}

// Can the shape be launched at all (shared memory and registers)?
int resident_shape_ok(uint32_t max_n, const stab_tune &tune, const LaunchCfg &lc) {
    const uint32_t G = tune.group_threads, tpc = tune.tableaux_per_cta;
    if (!G || !tpc || G * tpc > 1024 || (G != 32 && tpc > 15)) return 0;
    if (4 * res_words(max_n) * tpc > lc.smem_optin) return 0;
    cudaFuncAttributes fa{};
    cudaError_t e = tune.words_per_thread == 1 ? cudaFuncGetAttributes(&fa, k_resident<1>)
                  : tune.words_per_thread == 2 ? cudaFuncGetAttributes(&fa, k_resident<2>)
                                               : cudaFuncGetAttributes(&fa, k_resident<4>);
    if (e != cudaSuccess) { cudaGetLastError(); return 0; }
    const uint32_t regs = (uint32_t)fa.numRegs, thr = G * tpc;
    // registers are allocated per warp in units of 256
    const uint32_t per_warp = ((regs * 32 + 255) / 256) * 256;
    return per_warp * (thr / 32) <= 65536u && thr <= (uint32_t)fa.maxThreadsPerBlock;
}

cudaError_t resident_run(const ResJob *d_jobs, uint32_t n_jobs, uint32_t max_n, const stab_tune &tune,
                         unsigned int *d_counter, int *d_err, const LaunchCfg &lc, cudaStream_t s,
                         KernelProf *kp) {
    const uint32_t G = tune.group_threads, tpc = tune.tableaux_per_cta;
    const size_t gw = res_words(max_n);
    const size_t smem = 4 * gw * tpc;
    if (!resident_shape_ok(max_n, tune, lc)) return cudaErrorInvalidConfiguration;
    cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), s);
    int occ = 0;
    cudaError_t e = cudaSuccess;
    auto launch = [&](auto kern, int slot) {
        smem_attr_once(8 + slot, (const void *)kern, (int)lc.smem_optin);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (int)(G * tpc), smem);
        if (occ < 1) occ = 1;
        uint32_t groups_needed = (n_jobs + tpc - 1) / tpc;
        uint32_t grid = std::min<uint32_t>((uint32_t)(occ * lc.sm_count), std::max<uint32_t>(1, groups_needed));
        KernelProf::Rec rec;
        const bool timed = kp && (kp->mask & (1u << STAB_KERNEL_RESIDENT));
        if (kp) kp->launches++;
        if (timed) kp->begin(STAB_KERNEL_RESIDENT, s, rec);
        kern<<<grid, G * tpc, smem, s>>>(d_jobs, n_jobs, d_counter, d_err, G, (uint32_t)gw);
        if (timed) kp->end(rec, s, 0.0);
        e = cudaGetLastError();
    };
    switch (tune.words_per_thread) {
    case 1: launch(k_resident<1>, 1); break;
    case 2: launch(k_resident<2>, 2); break;
    default: launch(k_resident<4>, 4); break;
    }
    return e;
}

}  // namespace stab

// ---------------------------------------------------------------------------
// Allocation-free batch launch
// ---------------------------------------------------------------------------
// The resident engine's global scratch is its job table and its work counter.
// stab_sample_batch_noalloc keeps both in this file-scope device array instead
// of memory obtained from cudaMalloc.  Every GPU that loads the library holds
// the array until the process exits; all calls share it.  The job table is
// written on the device by k_noalloc_jobs from a by-value table of the call's
// groups (a kernel parameter), so no host staging buffer and no host-to-device
// copy is involved.
namespace stab {

constexpr uint32_t NOALLOC_MAX_SHOTS = 8192;
constexpr uint32_t NOALLOC_MAX_GROUPS = 64;
constexpr size_t NOALLOC_JOBS_OFF = 256;        // counter in the first 256 bytes
constexpr size_t NOALLOC_BYTES = NOALLOC_JOBS_OFF + (size_t)NOALLOC_MAX_SHOTS * sizeof(ResJob);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoallocGroup {           // one group with at least one shot
    const DevProg *prog;
    DevStreams st;
    unsigned long long *record;
    unsigned long long rec_stride;
    uint32_t first_job, shots;
};
struct NoallocTable {
    uint32_t n_groups, n_jobs;
    NoallocGroup g[NOALLOC_MAX_GROUPS];
};
static_assert(sizeof(NoallocTable) < 32000, "the group table must fit the kernel parameter space");

// Job k of the table: shot (k - first_job) of the group whose range holds k.
__global__ void k_noalloc_jobs(ResJob *jobs, const __grid_constant__ NoallocTable tab) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < tab.n_jobs; k += gridDim.x * blockDim.x) {
        uint32_t gi = 0;
        while (gi + 1 < tab.n_groups && tab.g[gi + 1].first_job <= k) gi++;
        const NoallocGroup &G = tab.g[gi];
        ResJob j;
        j.prog = G.prog;
        j.st = G.st;
        j.record = G.record;
        j.rec_stride = G.rec_stride;
        j.shot = k - G.first_job;
        j.pad = 0;
        jobs[k] = j;
    }
}

constexpr int NOALLOC_MAX_DEVICES = 64;
static void *g_noalloc_dev[NOALLOC_MAX_DEVICES];   // device address of the array, per device
static std::mutex g_noalloc_mu;

}  // namespace stab

extern "C" int stab_sample_batch_noalloc(stab_ctx *ctx, const stab_job_group *groups, size_t n_groups) {
    using namespace stab;
    if (!ctx) return fail(STAB_ERR_ARG, "context is NULL");
    if (n_groups && !groups) return fail(STAB_ERR_ARG, "groups is NULL");
    if (n_groups > NOALLOC_MAX_GROUPS)
        return fail(STAB_ERR_UNSUPPORTED, "stab_sample_batch_noalloc takes at most " +
                                              std::to_string(NOALLOC_MAX_GROUPS) + " groups");
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::lock_guard<std::mutex> lk2(g_noalloc_mu);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e) return cuda_fail(e, "cudaSetDevice");
    if (ctx->device < 0 || ctx->device >= NOALLOC_MAX_DEVICES)
        return fail(STAB_ERR_UNSUPPORTED, "device index too large for the allocation-free path");
    // set-up, once per device with that device current: the array's device address
    if (!g_noalloc_dev[ctx->device]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        g_noalloc_dev[ctx->device] = ptr;
    }
    unsigned char *base = (unsigned char *)g_noalloc_dev[ctx->device];
    // validate and size the batch before touching the device
    uint64_t total = 0;
    uint32_t max_n = 0;
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
        total += G.shots;
        max_n = std::max(max_n, p->n);
    }
    if (total > NOALLOC_MAX_SHOTS)
        return fail(STAB_ERR_UNSUPPORTED, "stab_sample_batch_noalloc runs at most " +
                                              std::to_string(NOALLOC_MAX_SHOTS) + " shots per call (got " +
                                              std::to_string(total) + ")");
    if (!total) return STAB_OK;
    // group table in decreasing cost order (longest shots first), on the stack
    uint32_t order[NOALLOC_MAX_GROUPS];
    uint64_t cost[NOALLOC_MAX_GROUPS];
    for (size_t gi = 0; gi < n_groups; gi++) {          // insertion sort: no temporary buffers
        const uint64_t c = find_prog(ctx, groups[gi].circuit_id)->cost;
        size_t j = gi;
        while (j > 0 && cost[j - 1] < c) {
            order[j] = order[j - 1];
            cost[j] = cost[j - 1];
            j--;
        }
        order[j] = (uint32_t)gi;
        cost[j] = c;
    }
    NoallocTable tab;
    memset(static_cast<void *>(&tab), 0, sizeof tab);
    for (size_t oi = 0; oi < n_groups; oi++) {
        const stab_job_group &G = groups[order[oi]];
        if (!G.shots) continue;
        NoallocGroup &T = tab.g[tab.n_groups++];
        T.prog = prog_desc(*find_prog(ctx, G.circuit_id));
        T.st = to_dev(G.streams);
        T.record = (unsigned long long *)G.d_record;
        T.rec_stride = G.record_words;
        T.first_job = tab.n_jobs;
        T.shots = G.shots;
        tab.n_jobs += G.shots;
        e = cudaMemsetAsync(G.d_record, 0, (size_t)G.shots * G.record_words * 8, ctx->stream);
        if (e) return cuda_fail(e, "clearing records");
    }
    ResJob *jobs = (ResJob *)(base + NOALLOC_JOBS_OFF);
    k_noalloc_jobs<<<(tab.n_jobs + 255) / 256, 256, 0, ctx->stream>>>(jobs, tab);
    e = cudaGetLastError();
    if (e) return cuda_fail(e, "writing the job table");
    const stab_tune t = lookup_tune(ctx, max_n);
    // resident_run zeroes the counter (first word of the array) before the launch
    e = resident_run(jobs, tab.n_jobs, max_n, t, (unsigned int *)base, ctx->d_err, ctx->lc, ctx->stream, nullptr);
    if (e) return cuda_fail(e, "resident launch");
    return STAB_OK;
}
