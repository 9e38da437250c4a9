/*
 * oracle/chp.c -- plain CPU Aaronson-Gottesman (CHP) stabilizer-tableau
 * simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never does.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper section / table / algorithm it follows):
 *  - Tableau (Sec. 2.3, "The CHP Formalism"): 2n rows, rows 0..n-1 are the
 *    destabilizers, rows n..2n-1 the stabilizers, each row x[0..n-1],
 *    z[0..n-1] and a sign bit r; row 2n is the scratch row.  Rows are stored
 *    as packed 64-bit words (row-major) but every operation below reads and
 *    writes one bit at a time, in plain loops.
 *  - Gates (Sec. 2.4, Table "Clifford gates and their bit operations"), on
 *    every row, using the pre-gate bits:
 *      H:  r ^= x_a z_a, swap x_a and z_a
 *      S:  r ^= x_a z_a, z_a ^= x_a
 *      CX: r ^= x_c z_t (x_t ^ z_c ^ 1), x_t ^= x_c, z_c ^= z_t
 *    The table prints the CX phase as x_c z_t; the full Aaronson-Gottesman
 *    term is used (reading recorded in the design notes).  Derived gates
 *    (Sec. 2.4 "Other Clifford gates can be derived"): X: r ^= z_a;
 *    Z: r ^= x_a; Y: r ^= x_a ^ z_a; CZ = H_b CX H_b gives
 *    r ^= x_a x_b (z_a ^ z_b), z_a ^= x_b, z_b ^= x_a; SWAP exchanges columns.
 *  - rowsum(h, i) and g (Appendix B, Alg. "rowsum"): sum = 2 r_h + 2 r_i +
 *    sum_j g(x_ij, z_ij, x_hj, z_hj); r_h = 0 if sum = 0 mod 4, 1 if 2 mod 4
 *    (left unchanged otherwise); then row h ^= row i.
 *  - Z measurement of qubit a (Sec. 2.4 measurement rules, Table row "Measure"):
 *    p = first stabilizer row with x_{p,a} = 1.  If it exists the outcome is
 *    random: rowsum(i, p) for every row i != p with x_{i,a} = 1; row p-n <-
 *    row p; row p <- +Z_a; r_p <- the coin.  Otherwise it is deterministic:
 *    scratch <- 0, rowsum(scratch, i+n) for each destabilizer i with
 *    x_{i,a} = 1 in ascending order; the outcome is r_scratch.
 *  - Reset: measure (consuming its coin slot), then X_a if the outcome is 1.
 *  - Commutation of a Pauli P = (x_P, z_P) with a row S (Sec. 3.2, the
 *    tableau-wide commutation equation): S anticommutes with P iff
 *    sum_j (x_P,j z_S,j + z_P,j x_S,j) is odd.  chp_commute evaluates it for
 *    every row of the tableau, one bit at a time.
 *  - Pauli-product measurement MPP of P (the measurement rules of Sec. 2.4
 *    with Z_a replaced by P, the commutation test above deciding which rows
 *    take part): p = first stabilizer row anticommuting with P.  If it exists
 *    the outcome is random: rowsum(i, p) for every other row i anticommuting
 *    with P; row p-n <- row p; row p <- P with sign r_p = the coin.  Otherwise
 *    scratch <- 0, rowsum(scratch, i+n) for each destabilizer i anticommuting
 *    with P (ascending i); the product must be +-P and the outcome is
 *    r_scratch.  Factors are X (x=1), Y (x=z=1), Z (z=1) on distinct qubits.
 *  - Pauli noise (Sec. 2.7, stochastic Pauli channels): a Pauli P on qubit a
 *    flips r on the rows it anticommutes with: X -> z_a, Z -> x_a, Y -> x_a^z_a.
 *    Draw semantics (one uint32 u per noise op): T = floor(p * 2^32);
 *      DEPOLARIZE1(p): error iff u < T, Pauli index (u*3)/T -> X, Y, Z;
 *      DEPOLARIZE2(p): error iff u < T, m = (u*15)/T + 1, Pauli m/4 on q0 and
 *                      m%4 on q1 (0 I, 1 X, 2 Y, 3 Z);
 *      PAULI_CHANNEL_1(px,py,pz): X if u < Tx, Y if u < Tx+Ty, Z if u < Tx+Ty+Tz.
 *      RESET_ERROR(gamma, q): three draws u0,u1,u2: if u0 < T(gamma) reset the
 *      qubit with coin (u1 & 1); then Z if u2 < T(q).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

enum {
    K_NOP = 0, K_H = 1, K_S = 2, K_X = 3, K_Y = 4, K_Z = 5, K_CX = 6, K_CZ = 7,
    K_SWAP = 8, K_M = 9, K_R = 10, K_DEP1 = 11, K_DEP2 = 12, K_PC1 = 13,
    K_TICK = 14, K_RESET_ERR = 15, K_MPP = 16, K_PAULI = 17
};

enum {
    OR_OK = 0, OR_BAD_ARG = -1, OR_OOM = -2, OR_STREAM_SHORT = -4,
    OR_ODD_PHASE = -10, OR_BAD_DET = -11
};

typedef struct {
    uint8_t kind, rsv0;
    uint16_t rsv1;
    uint32_t q0, q1, arg;
} chp_op;

typedef struct {
    uint64_t n_meas_random, n_meas_det;   /* M and R measurements */
    uint64_t sum_A;                       /* rows rowsum'd by random measurements */
    uint64_t sum_K;                       /* rows accumulated by deterministic ones */
    uint64_t n_gates, n_noise_events;
} chp_stats;

typedef struct {
    uint32_t n, W;          /* qubits, 64-bit words per row */
    uint64_t *x, *z;        /* (2n+2) * W: 2n rows, scratch row 2n, Pauli row 2n+1 */
    uint8_t *r;             /* 2n+2 */
} chp_t;

static inline int bit(const uint64_t *row, uint32_t j) {
    return (int)((row[j >> 6] >> (j & 63)) & 1u);
}
static inline void setb(uint64_t *row, uint32_t j, int v) {
    uint64_t m = (uint64_t)1 << (j & 63);
    if (v) row[j >> 6] |= m; else row[j >> 6] &= ~m;
}
static inline uint64_t *XR(chp_t *s, uint32_t i) { return s->x + (size_t)i * s->W; }
static inline uint64_t *ZR(chp_t *s, uint32_t i) { return s->z + (size_t)i * s->W; }

void chp_reset(chp_t *s) {
    size_t rows = 2 * (size_t)s->n + 2;
    memset(s->x, 0, rows * s->W * sizeof(uint64_t));
    memset(s->z, 0, rows * s->W * sizeof(uint64_t));
    memset(s->r, 0, rows);
    for (uint32_t i = 0; i < s->n; i++) {
        setb(XR(s, i), i, 1);             /* destabilizer i = X_i */
        setb(ZR(s, s->n + i), i, 1);      /* stabilizer i = Z_i */
    }
}

chp_t *chp_new(uint32_t n) {
    chp_t *s = (chp_t *)calloc(1, sizeof(chp_t));
    if (!s) return NULL;
    s->n = n;
    s->W = (n + 63) / 64;
    if (s->W == 0) s->W = 1;
    size_t rows = 2 * (size_t)n + 2;
    s->x = (uint64_t *)calloc(rows * s->W, sizeof(uint64_t));
    s->z = (uint64_t *)calloc(rows * s->W, sizeof(uint64_t));
    s->r = (uint8_t *)calloc(rows, 1);
    if (!s->x || !s->z || !s->r) {
        free(s->x); free(s->z); free(s->r); free(s);
        return NULL;
    }
    chp_reset(s);
    return s;
}

void chp_free(chp_t *s) {
    if (!s) return;
    free(s->x); free(s->z); free(s->r); free(s);
}

uint32_t chp_words(const chp_t *s) { return s->W; }

/* Copy the 2n tableau rows out / in (row-major, W words per row). */
void chp_get(chp_t *s, uint64_t *x, uint64_t *z, uint8_t *r) {
    size_t rows = 2 * (size_t)s->n;
    memcpy(x, s->x, rows * s->W * sizeof(uint64_t));
    memcpy(z, s->z, rows * s->W * sizeof(uint64_t));
    memcpy(r, s->r, rows);
}
void chp_set(chp_t *s, const uint64_t *x, const uint64_t *z, const uint8_t *r) {
    size_t rows = 2 * (size_t)s->n;
    memcpy(s->x, x, rows * s->W * sizeof(uint64_t));
    memcpy(s->z, z, rows * s->W * sizeof(uint64_t));
    memcpy(s->r, r, rows);
}

/* Appendix B: g(x1, z1, x2, z2), the power of i contributed by one qubit when
 * the Pauli (x1,z1) multiplies (x2,z2). */
int chp_g(int x1, int z1, int x2, int z2) {
    if (x1 == 0 && z1 == 0) return 0;
    if (x1 == 1 && z1 == 1) return z2 - x2;
    if (x1 == 1 && z1 == 0) return z2 * (2 * x2 - 1);
    return x2 * (1 - 2 * z2);             /* x1 == 0, z1 == 1 */
}

/* Appendix B: rowsum(h, i).  Returns the sum mod 4 (0..3). */
static int rowsum(chp_t *s, uint32_t h, uint32_t i) {
    long long sum = 2 * (long long)s->r[h] + 2 * (long long)s->r[i];
    uint64_t *xh = XR(s, h), *zh = ZR(s, h), *xi = XR(s, i), *zi = ZR(s, i);
    for (uint32_t j = 0; j < s->n; j++)
        sum += chp_g(bit(xi, j), bit(zi, j), bit(xh, j), bit(zh, j));
    int m = (int)(((sum % 4) + 4) % 4);
    if (m == 0) s->r[h] = 0;
    else if (m == 2) s->r[h] = 1;
    for (uint32_t j = 0; j < s->n; j++) {
        setb(xh, j, bit(xi, j) ^ bit(xh, j));
        setb(zh, j, bit(zi, j) ^ bit(zh, j));
    }
    return m;
}

/* Apply a single-qubit Pauli (1 X, 2 Y, 3 Z) to qubit a. */
static void apply_pauli(chp_t *s, uint32_t a, int P) {
    uint32_t rows = 2 * s->n;
    for (uint32_t i = 0; i < rows; i++) {
        int xa = bit(XR(s, i), a), za = bit(ZR(s, i), a);
        int flip = 0;
        if (P == 1) flip = za;
        else if (P == 3) flip = xa;
        else if (P == 2) flip = xa ^ za;
        s->r[i] ^= (uint8_t)flip;
    }
}

static void gate(chp_t *s, int kind, uint32_t a, uint32_t b) {
    uint32_t rows = 2 * s->n;
    for (uint32_t i = 0; i < rows; i++) {
        uint64_t *x = XR(s, i), *z = ZR(s, i);
        int xa = bit(x, a), za = bit(z, a);
        int xb = bit(x, b), zb = bit(z, b);
        switch (kind) {
        case K_H:
            s->r[i] ^= (uint8_t)(xa & za);
            setb(x, a, za); setb(z, a, xa);
            break;
        case K_S:
            s->r[i] ^= (uint8_t)(xa & za);
            setb(z, a, za ^ xa);
            break;
        case K_X: s->r[i] ^= (uint8_t)za; break;
        case K_Z: s->r[i] ^= (uint8_t)xa; break;
        case K_Y: s->r[i] ^= (uint8_t)(xa ^ za); break;
        case K_CX: /* control a, target b */
            s->r[i] ^= (uint8_t)(xa & zb & (xb ^ za ^ 1));
            setb(x, b, xb ^ xa);
            setb(z, a, za ^ zb);
            break;
        case K_CZ:
            s->r[i] ^= (uint8_t)(xa & xb & (za ^ zb));
            setb(z, a, za ^ xb);
            setb(z, b, zb ^ xa);
            break;
        case K_SWAP:
            setb(x, a, xb); setb(x, b, xa);
            setb(z, a, zb); setb(z, b, za);
            break;
        default: break;
        }
    }
}

/* Z measurement of qubit a.  Returns outcome (0/1) or a negative error. */
static int measure(chp_t *s, uint32_t a, int coin, chp_stats *st) {
    uint32_t n = s->n;
    uint32_t p = 0;
    int found = 0;
    for (uint32_t i = n; i < 2 * n; i++)
        if (bit(XR(s, i), a)) { p = i; found = 1; break; }
    if (found) {
        uint64_t cntA = 0;
        for (uint32_t i = 0; i < 2 * n; i++) {
            if (i == p || !bit(XR(s, i), a)) continue;
            int m = rowsum(s, i, p);
            cntA++;
            /* Only the destabilizer paired with p anticommutes with row p;
             * every other product is Hermitian (even power of i). */
            if ((m & 1) && i != p - n) return OR_ODD_PHASE;
        }
        memcpy(XR(s, p - n), XR(s, p), s->W * sizeof(uint64_t));
        memcpy(ZR(s, p - n), ZR(s, p), s->W * sizeof(uint64_t));
        s->r[p - n] = s->r[p];
        memset(XR(s, p), 0, s->W * sizeof(uint64_t));
        memset(ZR(s, p), 0, s->W * sizeof(uint64_t));
        setb(ZR(s, p), a, 1);
        s->r[p] = (uint8_t)(coin & 1);
        if (st) { st->n_meas_random++; st->sum_A += cntA; }
        return coin & 1;
    }
    uint32_t sc = 2 * n;
    memset(XR(s, sc), 0, s->W * sizeof(uint64_t));
    memset(ZR(s, sc), 0, s->W * sizeof(uint64_t));
    s->r[sc] = 0;
    uint64_t cntK = 0;
    for (uint32_t i = 0; i < n; i++) {
        if (!bit(XR(s, i), a)) continue;
        int m = rowsum(s, sc, i + n);
        cntK++;
        if (m & 1) return OR_ODD_PHASE;
    }
    /* The accumulated product must be +-Z_a. */
    for (uint32_t j = 0; j < n; j++)
        if (bit(XR(s, sc), j) || bit(ZR(s, sc), j) != (j == a)) return OR_BAD_DET;
    if (st) { st->n_meas_det++; st->sum_K += cntK; }
    return s->r[sc];
}

/* Sec. 3.2: does row i anticommute with the Pauli held in row pr? */
static int anticommutes(chp_t *s, uint32_t i, uint32_t pr) {
    uint64_t *xs = XR(s, i), *zs = ZR(s, i), *xp = XR(s, pr), *zp = ZR(s, pr);
    int acc = 0;
    for (uint32_t j = 0; j < s->n; j++)
        acc += bit(xp, j) * bit(zs, j) + bit(zp, j) * bit(xs, j);
    return acc & 1;
}

/* Commutation of m Paulis (px, pz: m x W words, row-major) with every row of
 * the tableau: bit i of out[k * ((2n+63)/64) + i/64] = 1 iff row i
 * anticommutes with Pauli k. */
int chp_commute(chp_t *s, const uint64_t *px, const uint64_t *pz, size_t m, uint64_t *out) {
    uint32_t n = s->n, pr = 2 * n + 1;
    size_t ow = (2 * (size_t)n + 63) / 64;
    memset(out, 0, m * ow * sizeof(uint64_t));
    for (size_t k = 0; k < m; k++) {
        memcpy(XR(s, pr), px + k * s->W, s->W * sizeof(uint64_t));
        memcpy(ZR(s, pr), pz + k * s->W, s->W * sizeof(uint64_t));
        for (uint32_t i = 0; i < 2 * n; i++)
            if (anticommutes(s, i, pr)) out[k * ow + i / 64] |= (uint64_t)1 << (i % 64);
    }
    return OR_OK;
}

/* Measurement of the Pauli product held in row 2n+1 (sign +).  Returns the
 * outcome (0/1) or a negative error. */
static int measure_pauli(chp_t *s, int coin, chp_stats *st) {
    uint32_t n = s->n, pr = 2 * n + 1;
    uint32_t p = 0;
    int found = 0;
    for (uint32_t i = n; i < 2 * n; i++)
        if (anticommutes(s, i, pr)) { p = i; found = 1; break; }
    if (found) {
        uint64_t cntA = 0;
        for (uint32_t i = 0; i < 2 * n; i++) {
            if (i == p || !anticommutes(s, i, pr)) continue;
            int m = rowsum(s, i, p);
            cntA++;
            if ((m & 1) && i != p - n) return OR_ODD_PHASE;
        }
        memcpy(XR(s, p - n), XR(s, p), s->W * sizeof(uint64_t));
        memcpy(ZR(s, p - n), ZR(s, p), s->W * sizeof(uint64_t));
        s->r[p - n] = s->r[p];
        memcpy(XR(s, p), XR(s, pr), s->W * sizeof(uint64_t));
        memcpy(ZR(s, p), ZR(s, pr), s->W * sizeof(uint64_t));
        s->r[p] = (uint8_t)(coin & 1);
        if (st) { st->n_meas_random++; st->sum_A += cntA; }
        return coin & 1;
    }
    uint32_t sc = 2 * n;
    memset(XR(s, sc), 0, s->W * sizeof(uint64_t));
    memset(ZR(s, sc), 0, s->W * sizeof(uint64_t));
    s->r[sc] = 0;
    uint64_t cntK = 0;
    for (uint32_t i = 0; i < n; i++) {
        if (!anticommutes(s, i, pr)) continue;
        int m = rowsum(s, sc, i + n);
        cntK++;
        if (m & 1) return OR_ODD_PHASE;
    }
    for (uint32_t j = 0; j < n; j++)
        if (bit(XR(s, sc), j) != bit(XR(s, pr), j) || bit(ZR(s, sc), j) != bit(ZR(s, pr), j))
            return OR_BAD_DET;
    if (st) { st->n_meas_det++; st->sum_K += cntK; }
    return s->r[sc];
}

static inline uint64_t thr(double p) {
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)(p * 4294967296.0);    /* exact product, truncation = floor */
}

/* Run ops[0..n_ops) on the current state.  Coin/noise/record ordinals start at
 * zero for this call.  Returns 0 or a negative error. */
int chp_run(chp_t *s, const chp_op *ops, size_t n_ops,
            const double *params, size_t n_params,
            const uint64_t *coins, size_t coin_words,
            const uint32_t *noise, size_t noise_words,
            uint64_t *record, size_t record_words, chp_stats *st) {
    uint64_t m_ord = 0, c_ord = 0, l_ord = 0;
    if (record) memset(record, 0, record_words * sizeof(uint64_t));
    for (size_t k = 0; k < n_ops; k++) {
        const chp_op *o = &ops[k];
        uint32_t a = o->q0, b = o->q1;
        int kind = o->kind;
        int two = (kind == K_CX || kind == K_CZ || kind == K_SWAP || kind == K_DEP2);
        if (kind == K_NOP || kind == K_TICK) continue;
        if (kind == K_MPP) {
            /* a = number of factors; the next a ops are its PAULI factors */
            uint32_t pr = 2 * s->n + 1;
            if (a == 0 || a > s->n || k + (size_t)a >= n_ops)
                return OR_BAD_ARG;
            memset(XR(s, pr), 0, s->W * sizeof(uint64_t));
            memset(ZR(s, pr), 0, s->W * sizeof(uint64_t));
            for (uint32_t f = 1; f <= a; f++) {
                const chp_op *fo = &ops[k + f];
                uint32_t q = fo->q0, c = fo->q1;
                if (fo->kind != K_PAULI || q >= s->n || c < 1 || c > 3) return OR_BAD_ARG;
                if (bit(XR(s, pr), q) || bit(ZR(s, pr), q)) return OR_BAD_ARG;   /* repeated qubit */
                if (c == 1 || c == 2) setb(XR(s, pr), q, 1);
                if (c == 2 || c == 3) setb(ZR(s, pr), q, 1);
            }
            if ((c_ord >> 6) >= coin_words || (m_ord >> 6) >= record_words) return OR_STREAM_SHORT;
            int coin = (int)((coins[c_ord >> 6] >> (c_ord & 63)) & 1u);
            c_ord++;
            int out = measure_pauli(s, coin, st);
            if (out < 0) return out;
            if (out) record[m_ord >> 6] |= (uint64_t)1 << (m_ord & 63);
            m_ord++;
            k += a;
            continue;
        }
        if (kind > K_RESET_ERR) return OR_BAD_ARG;
        if (a >= s->n || (two && (b >= s->n || b == a))) return OR_BAD_ARG;
        switch (kind) {
        case K_H: case K_S: case K_X: case K_Y: case K_Z:
        case K_CX: case K_CZ: case K_SWAP:
            gate(s, kind, a, b);
            if (st) st->n_gates++;
            break;
        case K_M: case K_R: {
            if ((c_ord >> 6) >= coin_words) return OR_STREAM_SHORT;
            int coin = (int)((coins[c_ord >> 6] >> (c_ord & 63)) & 1u);
            c_ord++;
            int out = measure(s, a, coin, st);
            if (out < 0) return out;
            if (kind == K_M) {
                if ((m_ord >> 6) >= record_words) return OR_STREAM_SHORT;
                if (out) record[m_ord >> 6] |= (uint64_t)1 << (m_ord & 63);
                m_ord++;
            } else if (out) {
                apply_pauli(s, a, 1);
            }
            break;
        }
        case K_DEP1: case K_DEP2: case K_PC1: {
            if (l_ord >= noise_words) return OR_STREAM_SHORT;
            if (o->arg >= n_params) return OR_BAD_ARG;
            uint64_t u = noise[l_ord++];
            const double *pp = params + 3 * (size_t)o->arg;
            if (kind == K_PC1) {
                uint64_t tx = thr(pp[0]), ty = thr(pp[1]), tz = thr(pp[2]);
                int P = 0;
                if (u < tx) P = 1;
                else if (u < tx + ty) P = 2;
                else if (u < tx + ty + tz) P = 3;
                if (P) { apply_pauli(s, a, P); if (st) st->n_noise_events++; }
            } else {
                uint64_t T = thr(pp[0]);
                if (u < T) {
                    if (kind == K_DEP1) {
                        apply_pauli(s, a, (int)((u * 3) / T) + 1);
                    } else {
                        int m = (int)((u * 15) / T) + 1;
                        if (m / 4) apply_pauli(s, a, m / 4);
                        if (m % 4) apply_pauli(s, b, m % 4);
                    }
                    if (st) st->n_noise_events++;
                }
            }
            break;
        }
        case K_RESET_ERR: {
            if (l_ord + 3 > noise_words) return OR_STREAM_SHORT;
            if (o->arg >= n_params) return OR_BAD_ARG;
            const double *pp = params + 3 * (size_t)o->arg;
            uint64_t u0 = noise[l_ord], u1 = noise[l_ord + 1], u2 = noise[l_ord + 2];
            l_ord += 3;
            if (u0 < thr(pp[0])) {
                int out = measure(s, a, (int)(u1 & 1u), st);
                if (out < 0) return out;
                if (out) apply_pauli(s, a, 1);
                if (st) st->n_noise_events++;
            }
            if (u2 < thr(pp[1])) { apply_pauli(s, a, 3); if (st) st->n_noise_events++; }
            break;
        }
        default:
            return OR_BAD_ARG;
        }
    }
    return OR_OK;
}

/* ---- many independent shots (fresh |0..0> each), split over threads ---- */
typedef struct {
    uint32_t n;
    const chp_op *ops; size_t n_ops;
    const double *params; size_t n_params;
    const uint64_t *coins; size_t coin_words;
    const uint32_t *noise; size_t noise_words;
    uint64_t *record; size_t record_words;
    uint64_t s0, s1;
    int status;
    chp_stats st;
} shot_job;

static void *shot_worker(void *arg) {
    shot_job *j = (shot_job *)arg;
    chp_t *s = chp_new(j->n);
    if (!s) { j->status = OR_OOM; return NULL; }
    for (uint64_t shot = j->s0; shot < j->s1; shot++) {
        chp_reset(s);
        int rc = chp_run(s, j->ops, j->n_ops, j->params, j->n_params,
                         j->coins + shot * j->coin_words, j->coin_words,
                         j->noise + shot * j->noise_words, j->noise_words,
                         j->record + shot * j->record_words, j->record_words, &j->st);
        if (rc) { j->status = rc; break; }
    }
    chp_free(s);
    return NULL;
}

int chp_sample(uint32_t n, const chp_op *ops, size_t n_ops,
               const double *params, size_t n_params, uint64_t shots,
               const uint64_t *coins, size_t coin_words,
               const uint32_t *noise, size_t noise_words,
               uint64_t *record, size_t record_words, int threads, chp_stats *st) {
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > shots) threads = shots ? (int)shots : 1;
    shot_job *jobs = (shot_job *)calloc((size_t)threads, sizeof(shot_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return OR_OOM; }
    for (int t = 0; t < threads; t++) {
        shot_job *j = &jobs[t];
        j->n = n; j->ops = ops; j->n_ops = n_ops; j->params = params; j->n_params = n_params;
        j->coins = coins; j->coin_words = coin_words; j->noise = noise;
        j->noise_words = noise_words; j->record = record; j->record_words = record_words;
        j->s0 = shots * (uint64_t)t / (uint64_t)threads;
        j->s1 = shots * (uint64_t)(t + 1) / (uint64_t)threads;
        if (threads == 1) shot_worker(j);
        else pthread_create(&tid[t], NULL, shot_worker, j);
    }
    int rc = OR_OK;
    for (int t = 0; t < threads; t++) {
        if (threads > 1) pthread_join(tid[t], NULL);
        if (jobs[t].status && !rc) rc = jobs[t].status;
        if (st) {
            st->n_meas_random += jobs[t].st.n_meas_random;
            st->n_meas_det += jobs[t].st.n_meas_det;
            st->sum_A += jobs[t].st.sum_A;
            st->sum_K += jobs[t].st.sum_K;
            st->n_gates += jobs[t].st.n_gates;
            st->n_noise_events += jobs[t].st.n_noise_events;
        }
    }
    free(jobs); free(tid);
    return rc;
}
