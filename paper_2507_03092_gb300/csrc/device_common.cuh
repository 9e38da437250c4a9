// device_common.cuh -- device helpers shared by the layered and resident
// engines: seeded streams, Clifford column rules, Pauli-noise decoding and the
// word-parallel rowsum phase.
#pragma once
#include "internal.h"

namespace stab {

#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------- streams
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output k of the stream with
// state s is mix64(s + (k+1) * G).
__device__ __forceinline__ unsigned long long sm_mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long sm_key(unsigned long long seed,
                                                      unsigned long long shot,
                                                      unsigned long long kind) {
    const unsigned long long G = 0x9E3779B97F4A7C15ull;
    return sm_mix64(sm_mix64(seed + kind * G) + (shot + 1) * G);
}
__device__ __forceinline__ unsigned long long sm_out(unsigned long long key,
                                                      unsigned long long k) {
    return sm_mix64(key + (k + 1) * 0x9E3779B97F4A7C15ull);
}

__device__ __forceinline__ uint32_t coin_bit(const DevStreams &s, uint32_t shot, uint32_t m) {
    unsigned long long w;
    if (s.mode == STAB_STREAM_SEEDED)
        w = sm_out(sm_key(s.seed, s.shot_offset + shot, 1ull), m >> 6);
    else
        w = s.coins[(unsigned long long)shot * s.coin_stride + (m >> 6)];
    return (uint32_t)((w >> (m & 63)) & 1ull);
}

__device__ __forceinline__ uint32_t noise_word(const DevStreams &s, uint32_t shot, uint32_t l) {
    if (s.mode == STAB_STREAM_SEEDED)
        return (uint32_t)(sm_out(sm_key(s.seed, s.shot_offset + shot, 2ull), l) >> 32);
    return s.noise[(unsigned long long)shot * s.noise_stride + l];
}

// ---------------------------------------------------------------- gates
// Column rules of Sec. 2.4 (Table) on one word of 32 rows, pre-gate bits;
// derived gates as in the op-kind documentation.  Returns the sign flips.
__device__ __forceinline__ uint32_t apply_gate(uint32_t g, uint32_t &xa, uint32_t &za,
                                               uint32_t &xb, uint32_t &zb) {
    uint32_t r = 0, t;
    switch (g) {
    case STAB_H: r = xa & za; t = xa; xa = za; za = t; break;
    case STAB_S: r = xa & za; za ^= xa; break;
    case STAB_X: r = za; break;
    case STAB_Y: r = xa ^ za; break;
    case STAB_Z: r = xa; break;
    case STAB_CX: r = xa & zb & ~(xb ^ za); xb ^= xa; za ^= zb; break;
    case STAB_CZ: r = xa & xb & (za ^ zb); za ^= xb; zb ^= xa; break;
    case STAB_SWAP: t = xa; xa = xb; xb = t; t = za; za = zb; zb = t; break;
    default: break;
    }
    return r;
}

// Sign flips from the Pauli P (1 X, 2 Y, 3 Z) on a column: rows that
// anticommute with P.
__device__ __forceinline__ uint32_t pauli_flip(int P, uint32_t x, uint32_t z) {
    return P == 1 ? z : P == 3 ? x : P == 2 ? (x ^ z) : 0u;
}

// Decode a noise draw: Pauli on the first target (pa) and second (pb).
__device__ __forceinline__ void noise_paulis(uint32_t kind, uint32_t u, const Thr &th,
                                             int &pa, int &pb) {
    pa = 0; pb = 0;
    unsigned long long uu = u;
    if (kind == STAB_PC1) {
        unsigned long long c = th.t[0];
        if (uu < c) { pa = 1; return; }
        c += th.t[1];
        if (uu < c) { pa = 2; return; }
        c += th.t[2];
        if (uu < c) pa = 3;
        return;
    }
    unsigned long long T = th.t[0];
    if (uu >= T) return;
    if (kind == STAB_DEP1) {
        pa = (int)((uu * 3ull) / T) + 1;
    } else {
        int m = (int)((uu * 15ull) / T) + 1;
        pa = m >> 2;
        pb = m & 3;
    }
}

// Apply item g's gate and noise to word values of columns a and b.
__device__ __forceinline__ uint32_t apply_item(const GItem &g, uint32_t &xa, uint32_t &za,
                                               uint32_t &xb, uint32_t &zb,
                                               const DevStreams &st, uint32_t shot,
                                               const Thr *thr) {
    uint32_t r = apply_gate(g.gate, xa, za, xb, zb);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        if (k >= g.nn) break;
        const uint32_t u = noise_word(st, shot, k ? g.nl[1] : g.nl[0]);
        int pa, pb;
        noise_paulis(k ? g.nk[1] : g.nk[0], u, thr[k ? g.np[1] : g.np[0]], pa, pb);
        if (!(pa | pb)) continue;
        int Pa = 0, Pb = 0;
        switch (k ? g.nt[1] : g.nt[0]) {
        case NT_A: Pa = pa; break;
        case NT_B: Pb = pa; break;
        case NT_AB: Pa = pa; Pb = pb; break;
        default: Pa = pb; Pb = pa; break;
        }
        r ^= pauli_flip(Pa, xa, za) ^ pauli_flip(Pb, xb, zb);
    }
    return r;
}

// ---------------------------------------------------------------- phase
// Power of i (mod 4) picked up on 32 qubits when the Pauli row (x1,z1)
// multiplies (x2,z2) from the left, word-parallel form of Appendix B's g:
// writing P(x,z) = i^{xz} X^x Z^z and commuting Z^{z1} past X^{x2} gives
// x1z1 + x2z2 + 2 z1x2 - x3z3 with x3 = x1^x2, z3 = z1^z2.
__device__ __forceinline__ int phase_word(uint32_t x1, uint32_t z1, uint32_t x2, uint32_t z2) {
    return __popc(x1 & z1) + __popc(x2 & z2) + 2 * __popc(z1 & x2) -
           __popc((x1 ^ x2) & (z1 ^ z2));
}

__device__ __forceinline__ void set_err(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// 32x32 bit transpose across a warp: lane i holds row i (bit j = column j);
// on return lane j holds column j (bit i = row i's bit j).  Stage s swaps the
// off-diagonal s x s blocks between lanes i and i ^ s: each lane keeps its
// half (mask m, or ~m in the upper lane of the pair) and sends the other half
// already moved into its partner's bit positions (a rotation by s, right in
// the lower lane and left in the upper one, masked), so a stage is a funnel
// shift, an AND, a shuffle and one three-input logic op.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v) {
    const int lane = threadIdx.x & 31;
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const int s = 16 >> k;
        const bool low = (lane & s) == 0;
        const uint32_t keep = low ? masks[k] : ~masks[k];
        const uint32_t send = __funnelshift_r(v, v, low ? s : 32 - s) & keep;
        v = (v & keep) | __shfl_xor_sync(FULL_MASK, send, s);
    }
    return v;
}

}  // namespace stab
