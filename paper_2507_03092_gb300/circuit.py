"""Circuit description and seeded circuit generators.

This module only *describes* circuits: the op record layout shared with the
C ABI (``include/stab.h``), a small builder, and the generators for the
synthetic workloads.  It simulates nothing and contains none of the tableau
arithmetic, so both the CUDA path and the CPU oracle consume its output.

Workloads (the paper measures only on generated circuits):

* rotated surface-code Z-memory (Sec. 2.5, "Planar surface code"; evaluation
  Sec. 4.1 "QEC Simulation"): data on a d x d grid, (d-1)^2 weight-4
  plaquettes in an X/Z checkerboard plus 2(d-1) weight-2 boundary checks,
  a 4-step CNOT schedule per round;
* random Clifford layers on n qubits with mid-circuit Z measurements;
* the random n-wide, n-round H/S/CX/M/R benchmark (Sec. 4.1, Fig. "random").

Noise channels are the stochastic Pauli channels of Sec. 2.7; the
Pauli-twirled T1/T2 probabilities (Sec. 2.7, twirling) are computed here on
the host because they are channel *parameters*, not simulation steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Op kinds -- must match enum stab_kind in include/stab.h.
NOP = 0
H = 1
S = 2
X = 3
Y = 4
Z = 5
CX = 6
CZ = 7
SWAP = 8
M = 9
R = 10
DEP1 = 11        # single-qubit depolarizing, params (p, 0, 0)
DEP2 = 12        # two-qubit depolarizing, params (p, 0, 0)
PC1 = 13         # single-qubit Pauli channel, params (px, py, pz)
TICK = 14        # layer hint; no effect on the state
RESET_ERR = 15   # composite relaxation/dephasing error, params (gamma, q, 0)
MPP = 16         # Pauli-product measurement: q0 = number of factors k, then k PAULI ops
PAULI = 17       # one factor of the preceding MPP: q0 = qubit, q1 = 1 X, 2 Y, 3 Z

KIND_NAMES = {
    NOP: "NOP", H: "H", S: "S", X: "X", Y: "Y", Z: "Z", CX: "CX", CZ: "CZ",
    SWAP: "SWAP", M: "M", R: "R", DEP1: "DEPOLARIZE1", DEP2: "DEPOLARIZE2",
    PC1: "PAULI_CHANNEL_1", TICK: "TICK", RESET_ERR: "RESET_ERROR", MPP: "MPP", PAULI: "PAULI",
}
ONE_QUBIT_GATES = (H, S, X, Y, Z)
TWO_QUBIT_GATES = (CX, CZ, SWAP)
NOISE_KINDS = (DEP1, DEP2, PC1, RESET_ERR)

# 16-byte op record, identical to struct stab_op.
OP_DTYPE = np.dtype([("kind", "<u1"), ("rsv0", "<u1"), ("rsv1", "<u2"),
                     ("q0", "<u4"), ("q1", "<u4"), ("arg", "<u4")])
assert OP_DTYPE.itemsize == 16


@dataclass
class Circuit:
    """A flat op list over ``n`` qubits plus its noise-parameter table."""

    n: int
    ops: np.ndarray                     # OP_DTYPE records
    params: np.ndarray                  # float64 [n_params, 3]
    meta: dict = field(default_factory=dict)

    @property
    def n_meas(self) -> int:            # record bits (M and MPP)
        k = self.ops["kind"]
        return int(np.count_nonzero((k == M) | (k == MPP)))

    @property
    def n_coin(self) -> int:            # coin slots (one per M, R or MPP)
        k = self.ops["kind"]
        return int(np.count_nonzero((k == M) | (k == R) | (k == MPP)))

    @property
    def n_noise(self) -> int:           # noise draws: one uint32 per noise op, three for RESET_ERROR
        k = self.ops["kind"]
        return int(np.count_nonzero(np.isin(k, (DEP1, DEP2, PC1)))
                   + 3 * np.count_nonzero(k == RESET_ERR))

    @property
    def record_words(self) -> int:
        return max(1, (self.n_meas + 63) // 64)

    @property
    def coin_words(self) -> int:
        return max(1, (self.n_coin + 63) // 64)

    @property
    def noise_words(self) -> int:
        return max(1, self.n_noise)

    def counts(self) -> dict:
        k = self.ops["kind"]
        return {KIND_NAMES[int(v)]: int(np.count_nonzero(k == v))
                for v in np.unique(k)}


class Builder:
    """Append-only op list with a de-duplicated parameter table."""

    def __init__(self, n: int):
        self.n = n
        self._ops: list[tuple] = []
        self._params: list[tuple] = []
        self._pidx: dict[tuple, int] = {}

    def _param(self, p: tuple) -> int:
        p = tuple(float(v) for v in (tuple(p) + (0.0, 0.0, 0.0))[:3])
        if p not in self._pidx:
            self._pidx[p] = len(self._params)
            self._params.append(p)
        return self._pidx[p]

    def op(self, kind: int, q0: int = 0, q1: int = 0, arg: int = 0):
        self._ops.append((kind, 0, 0, q0, q1, arg))
        return self

    def gate1(self, kind, q):
        return self.op(kind, q)

    def gate2(self, kind, a, b):
        return self.op(kind, a, b)

    def measure(self, q):
        return self.op(M, q)

    def reset(self, q):
        return self.op(R, q)

    def tick(self):
        return self.op(TICK)

    def dep1(self, q, p):
        return self.op(DEP1, q, 0, self._param((p,)))

    def dep2(self, a, b, p):
        return self.op(DEP2, a, b, self._param((p,)))

    def pauli_channel1(self, q, px, py, pz):
        return self.op(PC1, q, 0, self._param((px, py, pz)))

    def reset_error(self, q, gamma, qz):
        return self.op(RESET_ERR, q, 0, self._param((gamma, qz)))

    def mpp(self, factors):
        """Measure the Pauli product of ``factors`` [(qubit, 'X'|'Y'|'Z' or 1|2|3), ...]
        on distinct qubits; recorded like M."""
        code = {"X": 1, "Y": 2, "Z": 3}
        self.op(MPP, len(factors))
        for q, pch in factors:
            self.op(PAULI, int(q), code.get(pch, pch))
        return self

    def build(self, **meta) -> Circuit:
        ops = np.array(self._ops, dtype=OP_DTYPE) if self._ops else np.zeros(0, OP_DTYPE)
        params = (np.array(self._params, dtype=np.float64).reshape(-1, 3)
                  if self._params else np.zeros((0, 3), np.float64))
        return Circuit(self.n, ops, params, dict(meta))


# ---------------------------------------------------------------------------
# Rotated surface code (Sec. 2.5)
# ---------------------------------------------------------------------------

@dataclass
class SurfaceLayout:
    d: int
    n: int
    data: list           # data qubit index for (r, c): r*d + c
    plaquettes: list     # (pr, pc, 'X'|'Z', qubit index, [data corners in schedule order or None])
    x_anc: list
    z_anc: list


def surface_layout(d: int) -> SurfaceLayout:
    """Rotated code: data (r,c) in [0,d)^2; plaquette (pr,pc) covers the corners
    (pr,pc) NW, (pr,pc+1) NE, (pr+1,pc) SW, (pr+1,pc+1) SE that exist.
    Type X iff (pr+pc) is even.  Bulk plaquettes: 0<=pr,pc<=d-2.  Boundary:
    X on top (pr=-1) and bottom (pr=d-1), Z on left (pc=-1) and right (pc=d-1),
    kept only where the checkerboard gives that boundary's type.

    Schedule (4 CNOT steps): X checks visit NW, NE, SW, SE; Z checks visit
    NW, SW, NE, SE.  Every data qubit is visited by at most one check per step,
    and each X/Z pair of adjacent checks visits its two shared qubits in the
    same relative order, so the checks are measured without disturbing each
    other (pinned by the noiseless all-zero-detector test)."""
    if d < 2:
        raise ValueError("distance must be >= 2")
    nd = d * d
    plaq = []
    for pr in range(-1, d):
        for pc in range(-1, d):
            t = "X" if (pr + pc) % 2 == 0 else "Z"
            bulk = 0 <= pr <= d - 2 and 0 <= pc <= d - 2
            top = pr == -1 and 0 <= pc <= d - 2 and t == "X"
            bot = pr == d - 1 and 0 <= pc <= d - 2 and t == "X"
            left = pc == -1 and 0 <= pr <= d - 2 and t == "Z"
            right = pc == d - 1 and 0 <= pr <= d - 2 and t == "Z"
            if not (bulk or top or bot or left or right):
                continue
            corners = {"NW": (pr, pc), "NE": (pr, pc + 1),
                       "SW": (pr + 1, pc), "SE": (pr + 1, pc + 1)}
            order = ["NW", "NE", "SW", "SE"] if t == "X" else ["NW", "SW", "NE", "SE"]
            sched = []
            for key in order:
                r, c = corners[key]
                sched.append(r * d + c if (0 <= r < d and 0 <= c < d) else None)
            plaq.append([pr, pc, t, None, sched])
    for k, p in enumerate(plaq):
        p[3] = nd + k
    x_anc = [p[3] for p in plaq if p[2] == "X"]
    z_anc = [p[3] for p in plaq if p[2] == "Z"]
    return SurfaceLayout(d, nd + len(plaq), list(range(nd)),
                         [tuple(p) for p in plaq], x_anc, z_anc)


def surface_code_memory(d: int, rounds: int | None = None, p: float = 0.0,
                        t1t2: dict | None = None) -> Circuit:
    """Rotated surface-code Z-memory experiment.

    Reset every qubit; ``rounds`` syndrome rounds of
    (R ancillas, except in round 1) -> H on X ancillas -> 4 CNOT steps ->
    H on X ancillas -> M ancillas; then M every data qubit.
    Z checks use data->ancilla CNOTs, X checks ancilla->data CNOTs.

    Noise: ``p > 0`` adds DEPOLARIZE1(p) after every H and DEPOLARIZE2(p) after
    every CNOT.  ``t1t2`` (keys T1, T2, t1q, t2q, tm, all in the same time
    unit) adds PAULI_CHANNEL_1 with the twirled relaxation/dephasing
    probabilities after every op on its qubits, and on every qubit left idle in
    a layer for that layer's longest duration (reset takes the measurement
    duration)."""
    lay = surface_layout(d)
    rounds = d if rounds is None else rounds
    b = Builder(lay.n)
    allq = list(range(lay.n))
    anc = lay.x_anc + lay.z_anc
    anc_sorted = sorted(anc)

    def pc1(qs, dur):
        if t1t2 is None:
            return
        px, py, pz = twirled_pauli_probs(t1t2["T1"], t1t2["T2"], dur)
        for q in qs:
            b.pauli_channel1(q, px, py, pz)

    def idle(active, dur):
        if t1t2 is None:
            return
        act = set(active)
        pc1([q for q in allq if q not in act], dur)

    tm = t1t2["tm"] if t1t2 else 0.0
    t1q = t1t2["t1q"] if t1t2 else 0.0
    t2q = t1t2["t2q"] if t1t2 else 0.0

    # initial reset of every qubit
    for q in allq:
        b.reset(q)
    pc1(allq, tm)
    b.tick()
    meas_index = {}      # (round, ancilla) -> record ordinal
    rec = 0
    round_end = []       # op count at the end of each round (prefix lengths)
    for rd in range(rounds):
        if rd > 0:
            for q in anc_sorted:
                b.reset(q)
            pc1(anc_sorted, tm)
            idle(anc_sorted, tm)
            b.tick()
        for q in lay.x_anc:
            b.gate1(H, q)
            if p > 0:
                b.dep1(q, p)
        pc1(lay.x_anc, t1q)
        idle(lay.x_anc, t1q)
        b.tick()
        for step in range(4):
            active = []
            for (_pr, _pc, t, aq, sched) in lay.plaquettes:
                dq = sched[step]
                if dq is None:
                    continue
                c, tq = (aq, dq) if t == "X" else (dq, aq)
                b.gate2(CX, c, tq)
                if p > 0:
                    b.dep2(c, tq, p)
                if t1t2 is not None:
                    pc1([c, tq], t2q)
                active += [c, tq]
            idle(active, t2q)
            b.tick()
        for q in lay.x_anc:
            b.gate1(H, q)
            if p > 0:
                b.dep1(q, p)
        pc1(lay.x_anc, t1q)
        idle(lay.x_anc, t1q)
        b.tick()
        for q in anc_sorted:
            b.measure(q)
            meas_index[(rd, q)] = rec
            rec += 1
        pc1(anc_sorted, tm)
        idle(anc_sorted, tm)
        b.tick()
        round_end.append(len(b._ops))
    data_index = {}
    for q in lay.data:
        b.measure(q)
        data_index[q] = rec
        rec += 1
    c = b.build(kind="surface_code_memory", d=d, rounds=rounds, p=p,
                t1t2=t1t2, layout=lay, round_end=round_end)
    c.meta["detectors"] = surface_detectors(lay, rounds, meas_index, data_index)
    c.meta["observable"] = [data_index[q] for q in range(d)]   # Z along row 0
    return c


def surface_code_mpp(d: int, rounds: int | None = None, p: float = 0.0) -> Circuit:
    """Rotated surface-code Z-memory measured by Pauli products (the
    lattice-surgery view of Sec. 2.8): d*d data qubits only, every check
    measured directly as one MPP of its 2 or 4 corners.

    Reset the data; ``rounds`` rounds of DEPOLARIZE1(p) on every data qubit
    (``p > 0``) then MPP of every X check and every Z check (plaquette order of
    ``surface_layout``); then M every data qubit.  Detectors: Z checks in
    round 1, every check against the previous round, each Z check's final
    data parity against its last round."""
    lay = surface_layout(d)
    rounds = d if rounds is None else rounds
    nd = d * d
    b = Builder(nd)
    for q in range(nd):
        b.reset(q)
    b.tick()
    meas_index, rec = {}, 0
    for rd in range(rounds):
        if p > 0:
            for q in range(nd):
                b.dep1(q, p)
        for k, (_pr, _pc, t, _aq, sched) in enumerate(lay.plaquettes):
            b.mpp([(dq, t) for dq in sched if dq is not None])
            meas_index[(rd, k)] = rec
            rec += 1
        b.tick()
    data_index = {}
    for q in range(nd):
        b.measure(q)
        data_index[q] = rec
        rec += 1
    dets = []
    for k, pl in enumerate(lay.plaquettes):
        if pl[2] == "Z":
            dets.append([meas_index[(0, k)]])
    for rd in range(1, rounds):
        for k in range(len(lay.plaquettes)):
            dets.append([meas_index[(rd, k)], meas_index[(rd - 1, k)]])
    for k, (_pr, _pc, t, _aq, sched) in enumerate(lay.plaquettes):
        if t == "Z":
            dets.append([data_index[dq] for dq in sched if dq is not None] + [meas_index[(rounds - 1, k)]])
    c = b.build(kind="surface_code_mpp", d=d, rounds=rounds, p=p)
    c.meta["detectors"] = dets
    c.meta["observable"] = [data_index[q] for q in range(d)]
    return c


def surface_detectors(lay: SurfaceLayout, rounds: int, meas_index: dict,
                      data_index: dict) -> list:
    """Record-bit sets whose parity is 0 in a noiseless Z-memory run:
    Z ancillas in round 1; every ancilla in round r vs round r-1; each Z check's
    final data parity vs its last-round ancilla outcome."""
    dets = []
    for q in lay.z_anc:
        dets.append([meas_index[(0, q)]])
    for rd in range(1, rounds):
        for q in sorted(lay.x_anc + lay.z_anc):
            dets.append([meas_index[(rd, q)], meas_index[(rd - 1, q)]])
    for (_pr, _pc, t, aq, sched) in lay.plaquettes:
        if t != "Z":
            continue
        bits = [data_index[dq] for dq in sched if dq is not None]
        bits.append(meas_index[(rounds - 1, aq)])
        dets.append(bits)
    return dets


def twirled_pauli_probs(T1: float, T2: float, t: float) -> tuple:
    """Pauli-twirl of amplitude damping (T1) plus dephasing (T2) over time t:
    px = py = (1 - e^{-t/T1})/4,  pz = (1 - e^{-t/T2})/2 - (1 - e^{-t/T1})/4."""
    a = 1.0 - math.exp(-t / T1)
    px = a / 4.0
    pz = (1.0 - math.exp(-t / T2)) / 2.0 - a / 4.0
    return (px, px, pz)


def composite_t1t2_probs(T1: float, T2: float, t: float) -> tuple:
    """Composite relaxation + dephasing channel E_phase(E_relax(rho)) (Sec. 4.2)
    written as a positive mixture of stochastic Clifford+reset operations:
    reset to |0> with probability gamma = 1 - e^{-t/T1} (this reproduces the
    amplitude-damping populations and leaves coherence factor 1-gamma), then Z
    with probability q chosen so that (1-gamma)(1-2q) = e^{-t/T2}, i.e.
    q = (1 - e^{-t(1/T2 - 1/T1)})/2.  q >= 0 exactly when T1 >= T2, the regime
    in which the paper states the composite distribution is positive."""
    if T2 > T1:
        raise ValueError("the positive composite channel needs T1 >= T2")
    gamma = 1.0 - math.exp(-t / T1)
    qz = (1.0 - math.exp(-t * (1.0 / T2 - 1.0 / T1))) / 2.0
    return (gamma, qz)


# ---------------------------------------------------------------------------
# Random circuits
# ---------------------------------------------------------------------------

def random_clifford_layers(n: int, layers: int, seed: int = 0,
                           meas_frac: float = 0.10) -> Circuit:
    """Per layer: a seeded random permutation pairs the qubits; each pair gets
    a 2-qubit gate with probability 1/2 (CX or CZ with probability 1/2 each,
    random orientation), otherwise each of its qubits independently gets H or
    S; then Z-measure a random ``meas_frac`` of the qubits (without
    replacement, ascending).  The numpy PCG64 stream seeded by ``seed`` defines
    the circuit."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = Builder(n)
    k = int(round(meas_frac * n))
    for _ in range(layers):
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            a, c = int(perm[i]), int(perm[i + 1])
            if rng.random() < 0.5:
                kind = CX if rng.random() < 0.5 else CZ
                if rng.random() < 0.5:
                    a, c = c, a
                b.gate2(kind, a, c)
            else:
                b.gate1(H if rng.random() < 0.5 else S, a)
                b.gate1(H if rng.random() < 0.5 else S, c)
        if n % 2 == 1:
            b.gate1(H if rng.random() < 0.5 else S, int(perm[-1]))
        b.tick()
        for q in sorted(rng.choice(n, size=k, replace=False).tolist()):
            b.measure(int(q))
        b.tick()
    return b.build(kind="random_clifford_layers", layers=layers, seed=seed)


def random_wide_benchmark(n: int, rounds: int | None = None, seed: int = 0) -> Circuit:
    """Sec. 4.1, Fig. "random": ``rounds`` (default n) rounds; in each round
    every qubit receives one gate drawn uniformly from {H, S, CX, M, R}; a CX
    pairs the qubit with a uniformly drawn partner (distinct)."""
    rounds = n if rounds is None else rounds
    rng = np.random.Generator(np.random.PCG64(seed))
    b = Builder(n)
    for _ in range(rounds):
        for q in range(n):
            g = int(rng.integers(5))
            if g == 0:
                b.gate1(H, q)
            elif g == 1:
                b.gate1(S, q)
            elif g == 2 and n > 1:
                t = int(rng.integers(n - 1))
                t = t + 1 if t >= q else t
                b.gate2(CX, q, t)
            elif g == 3:
                b.measure(q)
            else:
                b.reset(q)
        b.tick()
    return b.build(kind="random_wide_benchmark", rounds=rounds, seed=seed)


def random_small_circuit(n: int, n_ops: int, seed: int, noise: bool = True,
                         allow=(H, S, X, Y, Z, CX, CZ, SWAP, M, R), mpp: bool = False) -> Circuit:
    """Uniformly random op soup for differential tests (any op at any time)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = Builder(n)
    kinds = list(allow)
    if noise:
        kinds += [DEP1, DEP2, PC1]
    if mpp:
        kinds += [MPP] * 4
    for _ in range(n_ops):
        kind = kinds[int(rng.integers(len(kinds)))]
        if kind == MPP:
            k = int(rng.integers(1, min(n, 5) + 1))
            qs = rng.choice(n, size=k, replace=False)
            b.mpp([(int(q), int(rng.integers(1, 4))) for q in qs])
            continue
        a = int(rng.integers(n))
        c = a
        if n > 1:
            c = int(rng.integers(n - 1))
            c = c + 1 if c >= a else c
        if kind in TWO_QUBIT_GATES:
            if n < 2:
                continue
            b.gate2(kind, a, c)
        elif kind == DEP1:
            b.dep1(a, float(rng.choice([0.05, 0.3, 1.0])))
        elif kind == DEP2:
            if n < 2:
                continue
            b.dep2(a, c, float(rng.choice([0.05, 0.3, 1.0])))
        elif kind == PC1:
            b.pauli_channel1(a, 0.1, 0.2, 0.3)
        elif kind == M:
            b.measure(a)
        elif kind == R:
            b.reset(a)
        else:
            b.gate1(kind, a)
    return b.build(kind="random_small", seed=seed)


def ghz(n: int) -> Circuit:
    b = Builder(n)
    b.gate1(H, 0)
    for q in range(1, n):
        b.gate2(CX, q - 1, q)
    for q in range(n):
        b.measure(q)
    return b.build(kind="ghz")


def prefix(c: Circuit, n_ops: int) -> Circuit:
    """The first ``n_ops`` ops of ``c`` (same qubits and parameter table)."""
    return Circuit(c.n, c.ops[:n_ops].copy(), c.params, {"prefix_of": c.meta.get("kind"), "n_ops": n_ops})


def gate_measure_ops(c: Circuit) -> int:
    """Clifford gates plus M, R and MPP ops (noise channels, TICKs and MPP
    factors excluded)."""
    k = c.ops["kind"]
    return int(np.count_nonzero(np.isin(k, ONE_QUBIT_GATES + TWO_QUBIT_GATES + (M, R, MPP))))


def concat(circuits: list[Circuit]) -> Circuit:
    """Concatenate circuits over the same qubit count (param tables merged)."""
    n = circuits[0].n
    ops, params = [], []
    off = 0
    for c in circuits:
        if c.n != n:
            raise ValueError("qubit counts differ")
        o = c.ops.copy()
        isn = np.isin(o["kind"], NOISE_KINDS)
        o["arg"][isn] += off
        ops.append(o)
        params.append(c.params)
        off += len(c.params)
    return Circuit(n, np.concatenate(ops), np.concatenate(params).reshape(-1, 3), {})
