// compile.cpp -- circuit compiler: flat op list -> layers of disjoint ops.
//
// The paper's sim2d (Sec. 3.1.4) runs independent gates of pre-flagged chunks
// concurrently and notes that scheduling at run time did not pay off; here the
// chunking is done once, at compile time, exactly: an op joins the current
// layer iff it is of the same class (unitary/noise vs. measurement) and touches
// no qubit already used in the layer.  Noise ops directly following a gate on
// the same qubits are attached to that gate's item, so the ubiquitous
// "gate, then its noise channel" pattern does not split layers.
#include "internal.h"

#include <cmath>
#include <cstring>
#include <algorithm>

namespace stab {

static unsigned long long threshold(double p) {
    if (!(p > 0.0)) return 0ull;
    if (p >= 1.0) return 1ull << 32;
    return (unsigned long long)(p * 4294967296.0);   // exact scaling, truncation = floor
}

static bool is_gate(uint8_t k) { return k >= STAB_H && k <= STAB_SWAP; }
static bool is_two(uint8_t k) { return k == STAB_CX || k == STAB_CZ || k == STAB_SWAP || k == STAB_DEP2; }
static bool is_noise(uint8_t k) { return k == STAB_DEP1 || k == STAB_DEP2 || k == STAB_PC1; }
static bool is_meas_class(uint8_t k) { return k == STAB_M || k == STAB_R || k == STAB_RESET_ERR; }

// Order of one gate layer's items for the slice kernel, whose threads take 16
// consecutive items per half-warp and read each operand's 8-byte slot: aligned
// groups of 16 items whose first operands lie in 16 distinct bank pairs (slot
// mod 16), and whose second operands do too, as far as the layer allows.
// Greedy: per group, the bank pairs of the first operand in order of the items
// left in them, each taking an item whose second operand's bank pair is not
// yet used (the fullest such class); a group left short is filled with the
// items that add the fewest repeats.  Any order of a layer's items gives the
// same tableau, since they act on disjoint qubits.
static void bank_order(const GItem *g, uint32_t count, std::vector<uint32_t> &perm) {
    std::vector<uint32_t> cls[16][16];
    uint32_t deg[16] = {0};
    for (uint32_t i = 0; i < count; i++) {
        const uint32_t ca = gate_slot(g[i].a) & 15u, cb = gate_slot(g[i].b) & 15u;
        cls[ca][cb].push_back(i);
        deg[ca]++;
    }
    perm.clear();
    perm.reserve(count);
    while (perm.size() < count) {
        uint32_t order[16];
        for (uint32_t c = 0; c < 16; c++) order[c] = c;
        std::stable_sort(order, order + 16, [&](uint32_t x, uint32_t y) { return deg[x] > deg[y]; });
        uint32_t na[16] = {0}, nb[16] = {0}, got = 0;
        const uint32_t want = (uint32_t)std::min<size_t>(16, count - perm.size());
        for (uint32_t k = 0; k < 16 && got < want; k++) {
            const uint32_t ca = order[k];
            if (!deg[ca]) break;
            int best = -1;
            for (uint32_t cb = 0; cb < 16; cb++)
                if (!nb[cb] && !cls[ca][cb].empty() && (best < 0 || cls[ca][cb].size() > cls[ca][best].size()))
                    best = (int)cb;
            if (best < 0) continue;
            perm.push_back(cls[ca][best].back());
            cls[ca][best].pop_back();
            deg[ca]--; na[ca]++; nb[best]++; got++;
        }
        while (got < want) {
            int ba = -1, bb = -1;
            uint32_t bs = 0;
            size_t bl = 0;
            for (uint32_t ca = 0; ca < 16; ca++)
                for (uint32_t cb = 0; cb < 16; cb++) {
                    if (cls[ca][cb].empty()) continue;
                    const uint32_t sc = na[ca] + nb[cb];
                    if (ba < 0 || sc < bs || (sc == bs && cls[ca][cb].size() > bl)) {
                        ba = (int)ca; bb = (int)cb; bs = sc; bl = cls[ca][cb].size();
                    }
                }
            perm.push_back(cls[ba][bb].back());
            cls[ba][bb].pop_back();
            deg[ba]--; na[ba]++; nb[bb]++; got++;
        }
    }
}

// Pauli-product measurement as a Clifford conjugation (the PBC rewriting of
// Sec. 2.8: a measurement absorbs the Cliffords around it).  U maps the
// product P of the factors to +Z on the last factor's qubit t:
//   X factor: H (X -> Z);  Y factor: Z, S, H (Y -> -Y -> X -> Z);  Z: nothing;
//   then CX(q_i, t) for every other factor q_i (Z_i Z_t -> Z_t).
// Measuring P equals applying U, measuring Z_t and applying U^dag, since
// U^dag (I +- Z_t) U / 2 = (I +- P) / 2; U^dag is CX(q_i, t) again, then H
// for X factors and H, S for Y factors.  Records are identical to the direct
// rule's: a measurement's outcome depends only on the state and its coin.
static void expand_mpp(const stab_op *ops, size_t n_ops, std::vector<stab_op> &out) {
    out.clear();
    out.reserve(n_ops * 2);
    auto one = [&](uint8_t kind, uint32_t a, uint32_t b = 0) {
        stab_op o{};
        o.kind = kind; o.q0 = a; o.q1 = b;
        out.push_back(o);
    };
    for (size_t k = 0; k < n_ops; k++) {
        const stab_op &o = ops[k];
        if (o.kind != STAB_MPP) { out.push_back(o); continue; }
        const uint32_t nf = o.q0;
        const stab_op *f = ops + k + 1;
        const uint32_t t = f[nf - 1].q0;
        for (uint32_t i = 0; i < nf; i++) {
            if (f[i].q1 == 1) one(STAB_H, f[i].q0);
            else if (f[i].q1 == 2) { one(STAB_Z, f[i].q0); one(STAB_S, f[i].q0); one(STAB_H, f[i].q0); }
        }
        for (uint32_t i = 0; i + 1 < nf; i++) one(STAB_CX, f[i].q0, t);
        one(STAB_M, t);
        for (uint32_t i = nf - 1; i-- > 0;) one(STAB_CX, f[i].q0, t);
        for (uint32_t i = 0; i < nf; i++) {
            if (f[i].q1 == 1) one(STAB_H, f[i].q0);
            else if (f[i].q1 == 2) { one(STAB_H, f[i].q0); one(STAB_S, f[i].q0); }
        }
        k += nf;
    }
}

int compile_program(uint32_t n, const stab_op *ops, size_t n_ops, const double *params,
                    size_t n_params, HostProg &P, std::string *err) {
    if (n == 0) { *err = "n must be positive"; return STAB_ERR_ARG; }
    if (n_ops && !ops) { *err = "ops is NULL"; return STAB_ERR_ARG; }
    if (n_params && !params) { *err = "params is NULL"; return STAB_ERR_ARG; }
    P.n = n;
    P.H = (n + 31) / 32;
    P.CW = 2 * P.H;
    P.thr.resize(n_params ? n_params : 1);
    for (size_t i = 0; i < n_params; i++) {
        for (int k = 0; k < 3; k++) {
            double v = params[3 * i + k];
            if (!(v >= 0.0) || v > 1.0) {
                *err = "noise parameter row " + std::to_string(i) + " outside [0, 1]";
                return STAB_ERR_ARG;
            }
            P.thr[i].t[k] = threshold(v);
        }
    }
    // ---- validate ----
    bool has_mpp = false;
    for (size_t k = 0; k < n_ops; k++) {
        const stab_op &o = ops[k];
        if (o.kind > STAB_PAULI) { *err = "op " + std::to_string(k) + ": unknown kind"; return STAB_ERR_ARG; }
        if (o.kind == STAB_NOP || o.kind == STAB_TICK) continue;
        if (o.kind == STAB_PAULI) {
            *err = "op " + std::to_string(k) + ": PAULI outside the factor list of an MPP";
            return STAB_ERR_ARG;
        }
        if (o.kind == STAB_MPP) {
            const uint32_t nf = o.q0;
            if (nf < 1 || nf > 64 || nf > n || k + nf >= n_ops) {
                *err = "op " + std::to_string(k) + ": MPP needs 1..64 (and at most n) factors following it";
                return STAB_ERR_ARG;
            }
            for (uint32_t i = 1; i <= nf; i++) {
                const stab_op &f = ops[k + i];
                if (f.kind != STAB_PAULI || f.q0 >= n || f.q1 < 1 || f.q1 > 3) {
                    *err = "op " + std::to_string(k + i) + ": MPP factor must be PAULI with qubit < n and code 1..3";
                    return STAB_ERR_ARG;
                }
                for (uint32_t i2 = 1; i2 < i; i2++)
                    if (ops[k + i2].q0 == f.q0) {
                        *err = "op " + std::to_string(k + i) + ": MPP factors must be on distinct qubits";
                        return STAB_ERR_ARG;
                    }
            }
            has_mpp = true;
            k += nf;
            continue;
        }
        if (o.q0 >= n) { *err = "op " + std::to_string(k) + ": qubit out of range"; return STAB_ERR_ARG; }
        if (is_two(o.kind) && (o.q1 >= n || o.q1 == o.q0)) {
            *err = "op " + std::to_string(k) + ": two-qubit op needs two distinct qubits < n";
            return STAB_ERR_ARG;
        }
        if ((is_noise(o.kind) || o.kind == STAB_RESET_ERR) && o.arg >= n_params) {
            *err = "op " + std::to_string(k) + ": parameter row out of range";
            return STAB_ERR_ARG;
        }
        if (o.kind == STAB_PC1) {
            const double *pp = params + 3 * (size_t)o.arg;
            if (P.thr[o.arg].t[0] + P.thr[o.arg].t[1] + P.thr[o.arg].t[2] > (1ull << 32) ||
                pp[0] + pp[1] + pp[2] > 1.0 + 1e-12) {
                *err = "op " + std::to_string(k) + ": PAULI_CHANNEL_1 probabilities sum above 1";
                return STAB_ERR_ARG;
            }
        }
    }
    // ---- layer ----
    // Two open layers, one per class (unitary/noise items, measurement items).
    // An op joins the last layer of its class when every qubit it touches was
    // last used in an earlier layer; otherwise it starts a new layer of its
    // class at the end.  Ops on disjoint qubits commute, so the layered
    // program equals the op list: an op never moves before an earlier op on
    // one of its qubits, and measurement-class ops keep their circuit order
    // (each goes into the last measurement layer or a new one after it), which
    // keeps the coin each random outcome reads the one of the op list.
    struct LB {
        int type;
        std::vector<GItem> g;
        std::vector<MItem> m;
    };
    struct Ref {
        int32_t layer = -1, idx = -1;
    };
    std::vector<LB> lays;
    std::vector<int32_t> front(n, -1);   // layer of the last op on each qubit
    std::vector<Ref> last_g(n);          // gate/noise item of the last op on q (if it was one)
    // last_m[q]: the measurement item of the last op on q if that op was an M or R
    std::vector<Ref> last_m(n);
    int32_t last_gl = -1, last_ml = -1;  // the open (last) layer of each class
    uint64_t m_ord = 0, c_ord = 0, l_ord = 0, n_gates = 0, n_real = 0;
    auto gate_layer = [&](int32_t lb) {
        if (last_gl >= 0 && lb <= last_gl) return last_gl;
        lays.push_back(LB{LT_GATE, {}, {}});
        return last_gl = (int32_t)lays.size() - 1;
    };
    auto meas_layer = [&](int32_t lb) {
        if (last_ml >= 0 && lb <= last_ml) return last_ml;
        lays.push_back(LB{LT_MEAS, {}, {}});
        return last_ml = (int32_t)lays.size() - 1;
    };
    auto put_gate = [&](const GItem &g) {
        const int32_t L = gate_layer(std::max(front[g.a], front[g.b]) + 1);
        lays[L].g.push_back(g);
        const Ref r{L, (int32_t)lays[L].g.size() - 1};
        front[g.a] = front[g.b] = L;
        last_g[g.a] = last_g[g.b] = r;
        last_m[g.a] = last_m[g.b] = Ref{};
    };

    for (size_t k = 0; k < n_ops; k++) {
        const stab_op &o = ops[k];
        uint8_t kind = o.kind;
        if (kind == STAB_NOP || kind == STAB_TICK) continue;
        n_real++;
        if (kind == STAB_MPP) {
            const uint32_t nf = o.q0;
            int32_t lb = 0;
            for (uint32_t i = 1; i <= nf; i++) lb = std::max(lb, front[ops[k + i].q0] + 1);
            const int32_t L = meas_layer(lb);
            MItem m{};
            m.q = ops[k + nf].q0;
            m.coin = (uint32_t)c_ord++;
            m.rec = (uint32_t)m_ord++;
            m.flags = MF_MPP;
            m.nl = (uint32_t)P.mfactors.size();
            m.np = nf;
            for (uint32_t i = 1; i <= nf; i++) {
                const stab_op &f = ops[k + i];
                P.mfactors.push_back(f.q0 | (f.q1 << 30));
                front[f.q0] = L;
                last_g[f.q0] = Ref{};
                last_m[f.q0] = Ref{};
            }
            lays[L].m.push_back(m);
            k += nf;
            continue;
        }
        uint32_t a = o.q0, b = is_two(kind) ? o.q1 : o.q0;
        if (kind == STAB_R && last_m[a].layer >= 0) {
            // R right after M/R on the same qubit: deterministic, outcome = that
            // measurement's; fold it in as "X if the outcome was 1" (or drop it
            // after a reset, whose outcome is 0).  Its coin slot is still used up.
            MItem &prev = lays[last_m[a].layer].m[last_m[a].idx];
            if (!(prev.flags & (MF_RESET | MF_RESET_AFTER))) prev.flags |= MF_RESET_AFTER;
            c_ord++;
            continue;
        }
        if (is_meas_class(kind)) {
            const int32_t L = meas_layer(front[a] + 1);
            MItem m{};
            m.q = a;
            m.rec = 0xffffffffu;
            if (kind == STAB_RESET_ERR) {
                m.flags = MF_RESET_ERR;
                m.nl = (uint32_t)l_ord;
                m.np = o.arg;
                l_ord += 3;
            } else {
                m.coin = (uint32_t)c_ord++;
                if (kind == STAB_M) m.rec = (uint32_t)m_ord++;
                else m.flags = MF_RESET;
            }
            lays[L].m.push_back(m);
            front[a] = L;
            last_g[a] = Ref{};
            last_m[a] = kind != STAB_RESET_ERR ? Ref{L, (int32_t)lays[L].m.size() - 1} : Ref{};
            continue;
        }
        if (is_gate(kind)) {
            n_gates++;
            GItem g{};
            g.a = a; g.b = b; g.gate = kind;
            put_gate(g);
            continue;
        }
        // noise op: joins the item of the gate (or noise) that was the last op
        // on its qubits, applied after it, else an item of its own
        uint32_t nl = (uint32_t)l_ord++;
        const Ref ra = last_g[a], rb = last_g[b];
        if (ra.layer >= 0 && (b == a || (rb.layer == ra.layer && rb.idx == ra.idx))) {
            GItem &g = lays[ra.layer].g[ra.idx];
            if (g.nn < 2 && (b == a || (g.a != g.b && (a == g.a || a == g.b)))) {
                uint8_t t;
                if (b == a) t = (a == g.a) ? NT_A : NT_B;
                else t = (a == g.a) ? NT_AB : NT_BA;
                g.nk[g.nn] = kind; g.nt[g.nn] = t; g.nl[g.nn] = nl; g.np[g.nn] = o.arg;
                g.nn++;
                last_m[a] = last_m[b] = Ref{};
                continue;
            }
        }
        GItem g{};
        g.a = a; g.b = b; g.gate = 0; g.nn = 1;
        g.nk[0] = kind; g.nt[0] = (b == a) ? NT_A : NT_AB; g.nl[0] = nl; g.np[0] = o.arg;
        put_gate(g);
    }
    // flatten: items of each layer contiguous, layers in order
    for (const LB &lb : lays) {
        Layer L{};
        L.type = (uint32_t)lb.type;
        if (lb.type == LT_GATE) {
            L.first = (uint32_t)P.gitems.size();
            L.count = (uint32_t)lb.g.size();
            P.gitems.insert(P.gitems.end(), lb.g.begin(), lb.g.end());
        } else {
            L.first = (uint32_t)P.mitems.size();
            L.count = (uint32_t)lb.m.size();
            P.mitems.insert(P.mitems.end(), lb.m.begin(), lb.m.end());
        }
        if (L.count) P.layers.push_back(L);
    }
    // folded resets may have flagged items of layers closed earlier
    P.rand_learn = true;
    for (auto &L : P.layers)
        if (L.type == LT_MEAS) {
            L.has_cond = 0;
            for (uint32_t i = L.first; i < L.first + L.count; i++) {
                if (P.mitems[i].flags & (MF_RESET | MF_RESET_ERR | MF_RESET_AFTER)) L.has_cond = 1;
                if (P.mitems[i].flags & MF_RESET_ERR) P.rand_learn = false;   // resets drawn by noise
            }
        }
    if (m_ord > 0xfffffff0ull || c_ord > 0xfffffff0ull || l_ord > 0xfffffff0ull) {
        *err = "circuit too long (more than 2^32 measurements or noise draws)";
        return STAB_ERR_UNSUPPORTED;
    }
    if (n > 65535) {
        // the packed items below hold 16-bit slots; engines reject such n anyway
    }
    // ---- packed items, item -> layer map, noise-event capacities ----
    P.sitems.resize(P.gitems.size());
    P.sab.resize(P.gitems.size());
    P.item_layer.resize(P.gitems.size());
    uint32_t ev_total = 0;
    std::vector<uint32_t> perm;
    for (uint32_t l = 0; l < P.layers.size(); l++) {
        Layer &L = P.layers[l];
        L.ev_off = ev_total;
        L.ev_cap = 0;
        L.n_noisy = 0;
        L.uniform = 0;
        if (L.type != LT_GATE) continue;
        L.uniform = L.count ? P.gitems[L.first].gate : 0u;
        bank_order(P.gitems.data() + L.first, L.count, perm);
        for (uint32_t i = L.first; i < L.first + L.count; i++) {
            const GItem &g = P.gitems[i];
            const GItem &gp = P.gitems[L.first + perm[i - L.first]];
            P.sitems[i].ab = (gate_slot(gp.a) & 0xffffu) | ((gate_slot(gp.b) & 0xffffu) << 16);
            P.sitems[i].g = gp.gate;
            P.sab[i] = P.sitems[i].ab;
            P.item_layer[i] = l;
            if (g.nn) L.n_noisy++;
            if (g.gate != L.uniform) L.uniform = 0;
        }
        // room for the expected events with a wide margin; a layer whose events
        // overflow falls back to evaluating every draw in the slice kernel
        if (L.n_noisy) L.ev_cap = std::min<uint32_t>(2 * L.n_noisy, 64 + L.n_noisy / 8);
        ev_total += L.ev_cap;
    }
    P.dev.ev_total = ev_total;
    // ---- runs for the layered engine ----
    uint32_t max_meas = 0, max_g = 0, n_gl = 0, n_ml = 0;
    for (uint32_t l = 0; l < P.layers.size(); l++) {
        const Layer &L = P.layers[l];
        if (L.type == LT_MEAS) {
            P.runs.push_back(Run{LT_MEAS, l, l + 1, 0.0});
            max_meas = std::max(max_meas, L.count);
            n_ml++;
        } else {
            if (!P.runs.empty() && P.runs.back().type == LT_GATE && P.runs.back().l1 == l)
                P.runs.back().l1 = l + 1;
            else
                P.runs.push_back(Run{LT_GATE, l, l + 1, 0.0});
            max_g = std::max(max_g, L.count);
            n_gl++;
        }
    }
    // Algorithmic bytes of a gate run (per tableau): every column the run
    // touches has its x and z bits over the 2n rows read and written once, the
    // sign column is read and written once, and each noise op reads one 4-byte
    // draw.  (Column = 2n bits = n/4 bytes.)
    {
        std::vector<uint32_t> seen(n, 0xffffffffu);
        const double col_bytes = 2.0 * n / 8.0;
        for (uint32_t ri = 0; ri < P.runs.size(); ri++) {
            Run &R = P.runs[ri];
            if (R.type != LT_GATE) continue;
            uint64_t cols = 0, draws = 0;
            for (uint32_t l = R.l0; l < R.l1; l++) {
                const Layer &L = P.layers[l];
                for (uint32_t i = L.first; i < L.first + L.count; i++) {
                    const GItem &g = P.gitems[i];
                    if (seen[g.a] != ri) { seen[g.a] = ri; cols++; }
                    if (seen[g.b] != ri) { seen[g.b] = ri; cols++; }
                    draws += g.nn;
                }
            }
            R.alg_bytes = (double)cols * 2 * 2 * col_bytes + 2 * col_bytes + 4.0 * (double)draws;
        }
    }
    stab_circuit_info &I = P.info;
    memset(&I, 0, sizeof(I));
    I.n = n;
    I.n_layers = (uint32_t)P.layers.size();
    I.n_ops = n_real;
    I.n_gates = n_gates;
    I.n_meas = m_ord;
    I.n_coin = c_ord;
    I.n_noise_words = l_ord;
    I.record_words = std::max<uint64_t>(1, (m_ord + 63) / 64);
    I.coin_words = std::max<uint64_t>(1, (c_ord + 63) / 64);
    I.n_gate_layers = n_gl;
    I.n_meas_layers = n_ml;
    I.max_layer_meas = max_meas;
    uint32_t n_runs_gate = 0;
    for (auto &r : P.runs) n_runs_gate += r.type == LT_GATE;
    I.n_gate_runs = n_runs_gate;
    // work estimate: word-ops over the column-packed tableau
    P.cost = (uint64_t)P.CW * (P.gitems.size() + 4 * P.mitems.size()) + P.layers.size() * 64;
    P.dev.n = n; P.dev.H = P.H; P.dev.CW = P.CW;
    P.dev.n_layers = (uint32_t)P.layers.size();
    P.dev.record_words = (uint32_t)I.record_words;
    P.dev.coin_words = (uint32_t)I.coin_words;
    P.dev.noise_words = (uint32_t)std::max<uint64_t>(1, l_ord);
    P.dev.max_meas = max_meas;
    P.dev.max_gitems = max_g;
    P.dev.n_gitems = (uint32_t)P.gitems.size();
    P.dev.n_mitems = (uint32_t)P.mitems.size();
    P.dev.n_mfactors = (uint32_t)P.mfactors.size();
    if (has_mpp) {
        std::vector<stab_op> ex;
        expand_mpp(ops, n_ops, ex);
        P.lay = std::make_unique<HostProg>();
        int rc = compile_program(n, ex.data(), ex.size(), params, n_params, *P.lay, err);
        if (rc) return rc;
    }
    return STAB_OK;
}

}  // namespace stab
