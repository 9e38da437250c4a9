"""Brute-force statevector simulator used to pin the CHP oracle (n <= 10).

Independent of the tableau formalism: gates are unitary matrices acting on a
2^n complex vector; a Z measurement computes the Born probability of outcome
1, which for a stabilizer state is exactly 0, 1/2 or 1.  Random outcomes
(probability 1/2) take the coin; deterministic ones must not.  Noise draws use
the documented integer threshold rules.
"""
from __future__ import annotations

import numpy as np

from paper_2507_03092_gb300 import circuit as C

_SQ2 = 1 / np.sqrt(2)
MAT = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
    "H": np.array([[1, 1], [1, -1]], dtype=complex) * _SQ2,
    "S": np.array([[1, 0], [0, 1j]], dtype=complex),
}
PAULI_OF_CODE = {0: "I", 1: "X", 2: "Y", 3: "Z"}


class StateVector:
    def __init__(self, n: int):
        self.n = n
        self.psi = np.zeros(2 ** n, dtype=complex)
        self.psi[0] = 1.0

    def _axis_view(self, q):
        # reshape so that axis 1 is qubit q (little-endian qubit order)
        return self.psi.reshape(2 ** (self.n - q - 1), 2, 2 ** q)

    def apply1(self, U, q):
        v = self._axis_view(q)
        self.psi = np.einsum("ab,ibj->iaj", U, v).reshape(-1)

    def apply_cx(self, c, t):
        idx = np.arange(2 ** self.n)
        m = ((idx >> c) & 1) == 1
        src = idx ^ (1 << t)
        new = self.psi.copy()
        new[m] = self.psi[src[m]]
        self.psi = new

    def apply_cz(self, a, b):
        idx = np.arange(2 ** self.n)
        m = (((idx >> a) & 1) & ((idx >> b) & 1)) == 1
        self.psi[m] *= -1

    def apply_swap(self, a, b):
        idx = np.arange(2 ** self.n)
        ba, bb = (idx >> a) & 1, (idx >> b) & 1
        src = idx ^ ((ba ^ bb) << a) ^ ((ba ^ bb) << b)
        self.psi = self.psi[src]

    def prob1(self, q) -> float:
        idx = np.arange(2 ** self.n)
        return float(np.sum(np.abs(self.psi[((idx >> q) & 1) == 1]) ** 2))

    def measure(self, q, coin) -> tuple[int, bool]:
        """Returns (outcome, was_random)."""
        p1 = self.prob1(q)
        if abs(p1 - 0.5) < 1e-9:
            out, rnd = int(coin) & 1, True
        elif p1 < 1e-9:
            out, rnd = 0, False
        elif p1 > 1 - 1e-9:
            out, rnd = 1, False
        else:
            raise AssertionError(f"non-stabilizer probability {p1}")
        idx = np.arange(2 ** self.n)
        keep = ((idx >> q) & 1) == out
        self.psi = np.where(keep, self.psi, 0)
        self.psi /= np.linalg.norm(self.psi)
        return out, rnd

    def pauli(self, q, code):
        if code:
            self.apply1(MAT[PAULI_OF_CODE[code]], q)

    def apply_product(self, factors, psi):
        out = StateVector(self.n)
        out.psi = psi.copy()
        for q, code in factors:
            out.pauli(q, code)
        return out.psi

    def measure_product(self, factors, coin) -> tuple[int, bool]:
        """Projective measurement of the Hermitian Pauli product P: outcome 1
        (eigenvalue -1) has probability (1 - <psi|P|psi>)/2; the post-state
        is (psi +- P psi) normalised."""
        Ppsi = self.apply_product(factors, self.psi)
        ev = float(np.real(np.vdot(self.psi, Ppsi)))
        p1 = (1 - ev) / 2
        if abs(p1 - 0.5) < 1e-9:
            out, rnd = int(coin) & 1, True
        elif p1 < 1e-9:
            out, rnd = 0, False
        elif p1 > 1 - 1e-9:
            out, rnd = 1, False
        else:
            raise AssertionError(f"non-stabilizer probability {p1}")
        self.psi = self.psi + (1 - 2 * out) * Ppsi
        self.psi /= np.linalg.norm(self.psi)
        return out, rnd


def threshold(p: float) -> int:
    if not p > 0:
        return 0
    if p >= 1:
        return 1 << 32
    return int(p * 4294967296.0)


def run(circ: C.Circuit, coins, noise):
    """Returns (record bits list, list of (op index, was_random))."""
    sv = StateVector(circ.n)
    coins = np.asarray(coins, np.uint64).ravel()
    noise = np.asarray(noise, np.uint32).ravel()
    rec, rnd = [], []
    ci = li = 0
    skip = 0
    for k, o in enumerate(circ.ops):
        if skip:
            skip -= 1
            continue
        kind, a, b = int(o["kind"]), int(o["q0"]), int(o["q1"])
        pp = circ.params[int(o["arg"])] if kind in C.NOISE_KINDS else None
        if kind in (C.H, C.S, C.X, C.Y, C.Z):
            sv.apply1(MAT[C.KIND_NAMES[kind]], a)
        elif kind == C.CX:
            sv.apply_cx(a, b)
        elif kind == C.CZ:
            sv.apply_cz(a, b)
        elif kind == C.SWAP:
            sv.apply_swap(a, b)
        elif kind in (C.M, C.R):
            coin = (int(coins[ci >> 6]) >> (ci & 63)) & 1
            ci += 1
            out, r = sv.measure(a, coin)
            rnd.append((k, r))
            if kind == C.M:
                rec.append(out)
            elif out:
                sv.apply1(MAT["X"], a)
        elif kind == C.MPP:
            factors = [(int(f["q0"]), int(f["q1"])) for f in circ.ops[k + 1:k + 1 + a]]
            skip = a
            coin = (int(coins[ci >> 6]) >> (ci & 63)) & 1
            ci += 1
            out, r = sv.measure_product(factors, coin)
            rnd.append((k, r))
            rec.append(out)
        elif kind == C.DEP1:
            u, T = int(noise[li]), threshold(pp[0])
            li += 1
            if u < T:
                sv.pauli(a, (u * 3) // T + 1)
        elif kind == C.DEP2:
            u, T = int(noise[li]), threshold(pp[0])
            li += 1
            if u < T:
                m = (u * 15) // T + 1
                sv.pauli(a, m // 4)
                sv.pauli(b, m % 4)
        elif kind == C.PC1:
            u = int(noise[li])
            li += 1
            tx, ty, tz = (threshold(v) for v in pp)
            if u < tx:
                sv.pauli(a, 1)
            elif u < tx + ty:
                sv.pauli(a, 2)
            elif u < tx + ty + tz:
                sv.pauli(a, 3)
        elif kind == C.RESET_ERR:
            u0, u1, u2 = (int(v) for v in noise[li:li + 3])
            li += 3
            if u0 < threshold(pp[0]):
                out, _ = sv.measure(a, u1 & 1)
                if out:
                    sv.apply1(MAT["X"], a)
            if u2 < threshold(pp[1]):
                sv.pauli(a, 3)
    return rec, rnd
