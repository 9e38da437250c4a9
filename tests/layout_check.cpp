// Host-side check of the layered engine's packed gate layers (no GPU).
//
// Usage: layout_check OPS PARAMS N
//   OPS: the circuit's op records (16 bytes each, as stab_op), PARAMS: its
//   float64 parameter rows, N: qubits.
//
// Prints "slot ok" once gate_slot has been checked to permute every aligned
// block of 16 columns below 65536 and to be its own inverse; then, per gate
// layer, "layer <index> <items> <two-qubit> <now> <identity> <ideal>":
//   now      -- shared-memory wavefronts of the slice kernel's operand reads
//               in the packed order (8-byte slots, 16 per half-warp: each
//               aligned group of 16 items costs, per operand, the largest
//               number of distinct slots in one bank pair, slot mod 16),
//   identity -- the same for the layer's items in circuit order with the
//               column index as the slot,
//   ideal    -- one wavefront per group and operand.
// Exits non-zero if a layer's packed items are not its items, reordered,
// with their operands' slots and gate kinds.
#include "../paper_2507_03092_gb300/csrc/internal.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

using namespace stab;

static std::vector<unsigned char> read_file(const char *path) {
    std::vector<unsigned char> out;
    FILE *f = std::fopen(path, "rb");
    if (!f) return out;
    unsigned char buf[1 << 16];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) out.insert(out.end(), buf, buf + k);
    std::fclose(f);
    return out;
}

// wavefronts of one operand's reads: aligned groups of 16 items
static uint64_t wavefronts(const std::vector<uint32_t> &slots) {
    uint64_t tot = 0;
    for (size_t g = 0; g < slots.size(); g += 16) {
        std::vector<uint32_t> u(slots.begin() + g, slots.begin() + std::min(slots.size(), g + 16));
        std::sort(u.begin(), u.end());
        u.erase(std::unique(u.begin(), u.end()), u.end());
        uint32_t cnt[16] = {0}, mx = 0;
        for (uint32_t s : u) mx = std::max(mx, ++cnt[s & 15u]);
        tot += mx;
    }
    return tot;
}

int main(int argc, char **argv) {
    if (argc != 4) {
        std::fprintf(stderr, "usage: layout_check OPS PARAMS N\n");
        return 2;
    }
    for (uint32_t b = 0; b < 65536; b += 16) {
        bool seen[16] = {false};
        for (uint32_t j = b; j < b + 16; j++) {
            const uint32_t s = gate_slot(j);
            if (s < b || s >= b + 16 || seen[s - b] || gate_slot(s) != j) {
                std::fprintf(stderr, "gate_slot fails at column %u\n", j);
                return 1;
            }
            seen[s - b] = true;
        }
    }
    std::printf("slot ok\n");

    const std::vector<unsigned char> ob = read_file(argv[1]), pb = read_file(argv[2]);
    if (ob.size() % sizeof(stab_op) || pb.size() % (3 * sizeof(double))) {
        std::fprintf(stderr, "bad input sizes\n");
        return 2;
    }
    std::vector<stab_op> ops(ob.size() / sizeof(stab_op));
    if (!ops.empty()) std::memcpy(ops.data(), ob.data(), ob.size());
    std::vector<double> params(pb.size() / sizeof(double));
    if (!params.empty()) std::memcpy(params.data(), pb.data(), pb.size());
    HostProg P;
    std::string err;
    const int rc = compile_program((uint32_t)std::stoul(argv[3]), ops.data(), ops.size(), params.data(),
                                   params.size() / 3, P, &err);
    if (rc) {
        std::fprintf(stderr, "compile failed: %s\n", err.c_str());
        return 1;
    }
    for (uint32_t l = 0; l < P.layers.size(); l++) {
        const Layer &L = P.layers[l];
        if (L.type != LT_GATE) continue;
        std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> want, got;
        std::vector<uint32_t> na, nb, ia, ib;
        bool two = false;
        for (uint32_t i = L.first; i < L.first + L.count; i++) {
            const GItem &g = P.gitems[i];
            want.emplace_back(gate_slot(g.a), gate_slot(g.b), g.gate);
            const uint32_t a = P.sitems[i].ab & 0xffffu, b = P.sitems[i].ab >> 16;
            got.emplace_back(a, b, P.sitems[i].g);
            if (P.sab[i] != P.sitems[i].ab) {
                std::fprintf(stderr, "layer %u: the two packed copies differ\n", l);
                return 1;
            }
            na.push_back(a);
            nb.push_back(b);
            ia.push_back(g.a);
            ib.push_back(g.b);
            two = two || g.a != g.b;
        }
        std::sort(want.begin(), want.end());
        std::sort(got.begin(), got.end());
        if (want != got) {
            std::fprintf(stderr, "layer %u: packed items are not the layer's items\n", l);
            return 1;
        }
        const uint64_t now = wavefronts(na) + (two ? wavefronts(nb) : 0);
        const uint64_t idn = wavefronts(ia) + (two ? wavefronts(ib) : 0);
        const uint64_t ideal = (uint64_t)(two ? 2 : 1) * ((L.count + 15) / 16);
        std::printf("layer %u %u %d %llu %llu %llu\n", l, L.count, two ? 1 : 0, (unsigned long long)now,
                    (unsigned long long)idn, (unsigned long long)ideal);
    }
    return 0;
}
