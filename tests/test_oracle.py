"""Pins for the CPU oracle (oracle/chp.c) against things other than itself:
Pauli matrix algebra, unitary conjugation, brute-force statevector simulation,
closed-form circuits, tableau invariants and the noiseless surface-code
detectors.  No GPU."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2507_03092_gb300 import circuit as C
from paper_2507_03092_gb300 import streams as S
from tests import statevec as SV

P_OF = {(0, 0): "I", (1, 0): "X", (1, 1): "Y", (0, 1): "Z"}


def pauli_matrix(bits):
    return SV.MAT[P_OF[bits]]


# ---------------------------------------------------------------- g, f, phase

def test_g_is_power_of_i_in_pauli_products():
    """Appendix B: g(x1,z1,x2,z2) is the exponent e with P1 P2 = i^e P3."""
    for x1, z1, x2, z2 in itertools.product((0, 1), repeat=4):
        e = oracle.g(x1, z1, x2, z2)
        lhs = pauli_matrix((x1, z1)) @ pauli_matrix((x2, z2))
        rhs = (1j ** e) * pauli_matrix((x1 ^ x2, z1 ^ z2))
        assert np.allclose(lhs, rhs), (x1, z1, x2, z2, e)
        assert e in (-1, 0, 1)


def test_alg1_phase_polynomial_equals_g():
    """Alg. 1's branch-free polynomial is the same function as g."""
    def f(xp, zp, xh, zh):
        return xp * (zp * (zh - xh) + (1 - zp) * zh * (2 * xh - 1)) + (1 - xp) * zp * xh * (1 - 2 * zh)
    for args in itertools.product((0, 1), repeat=4):
        assert f(*args) == oracle.g(*args)


def test_word_parallel_phase_identity():
    """sum_j g over packed words == popc(x1&z1)+popc(x2&z2)+2popc(z1&x2)-popc(x3&z3)
    (mod 4): the identity the CUDA rowsum uses, checked on random words."""
    rng = np.random.default_rng(1)
    pc = lambda v: bin(v).count("1")
    for _ in range(300):
        x1, z1, x2, z2 = (int(v) for v in rng.integers(0, 2 ** 63, 4))
        ref = sum(oracle.g((x1 >> j) & 1, (z1 >> j) & 1, (x2 >> j) & 1, (z2 >> j) & 1)
                  for j in range(63))
        got = pc(x1 & z1) + pc(x2 & z2) + 2 * pc(z1 & x2) - pc((x1 ^ x2) & (z1 ^ z2))
        assert (ref - got) % 4 == 0


def test_ordered_product_closed_form():
    """Sign of an ordered product of commuting Paulis from the closed form
    2 sum r + sum popc(x_b&z_b) + 2 sum_{a<b} popc(z_a&x_b) - popc(X&Z) equals
    the sign obtained by multiplying the matrices (brute force, 3 qubits)."""
    rng = np.random.default_rng(7)
    pc = lambda v: bin(v).count("1")
    nq = 3

    def mat(x, z, r):
        M = np.array([[1.0 + 0j]])
        for j in reversed(range(nq)):
            M = np.kron(M, pauli_matrix(((x >> j) & 1, (z >> j) & 1)))
        return (-1) ** r * M

    for _ in range(200):
        k = int(rng.integers(1, 5))
        rows = [(int(rng.integers(0, 8)), int(rng.integers(0, 8)), int(rng.integers(0, 2)))
                for _ in range(k)]
        prod = np.eye(2 ** nq, dtype=complex)
        for x, z, r in rows:
            prod = prod @ mat(x, z, r)
        X = Z = 0
        e = 0
        for b, (x, z, r) in enumerate(rows):
            e += 2 * r + pc(x & z)
            for a in range(b):
                e += 2 * pc(rows[a][1] & x)
            X ^= x
            Z ^= z
        e -= pc(X & Z)
        assert np.allclose(prod, (1j ** e) * mat(X, Z, 0))


# ---------------------------------------------------------------- gate rules

def _gate_unitary(kind):
    U = np.zeros((4, 4), dtype=complex)
    for col in range(4):
        sv = SV.StateVector(2)
        sv.psi[:] = 0
        sv.psi[col] = 1
        if kind in (C.H, C.S, C.X, C.Y, C.Z):
            sv.apply1(SV.MAT[C.KIND_NAMES[kind]], 0)
        elif kind == C.CX:
            sv.apply_cx(0, 1)
        elif kind == C.CZ:
            sv.apply_cz(0, 1)
        elif kind == C.SWAP:
            sv.apply_swap(0, 1)
        U[:, col] = sv.psi
    return U


def _row_matrix(x, z, r):
    # qubit 1 is the more significant tensor factor
    return (-1) ** r * np.kron(pauli_matrix((int(x[1]), int(z[1]))),
                               pauli_matrix((int(x[0]), int(z[0]))))


@pytest.mark.parametrize("kind", [C.H, C.S, C.X, C.Y, C.Z, C.CX, C.CZ, C.SWAP])
def test_gate_rule_is_conjugation(kind):
    """Each tableau gate rule maps every signed 2-qubit Pauli P to U P U^dag
    (Sec. 2.4 Table; derived gates checked the same way)."""
    n = 16                            # 32 rows: every Pauli on qubits 0,1, both signs
    t = oracle.Tableau(n)
    x = np.zeros((2 * n, t.W), np.uint64)
    z = np.zeros((2 * n, t.W), np.uint64)
    r = np.zeros(2 * n, np.uint8)
    combos = list(itertools.product((0, 1), repeat=5))
    for i, (x0, z0, x1, z1, s) in enumerate(combos):
        x[i, 0] = x0 | (x1 << 1)
        z[i, 0] = z0 | (z1 << 1)
        r[i] = s
    t.set(x, z, r)
    b = C.Builder(n)
    if kind in C.TWO_QUBIT_GATES:
        b.gate2(kind, 0, 1)
    else:
        b.gate1(kind, 0)
    t.run(b.build())
    x2, z2, r2 = t.get()
    U = _gate_unitary(kind)
    for i, (x0, z0, x1, z1, s) in enumerate(combos):
        want = U @ _row_matrix((x0, x1), (z0, z1), s) @ U.conj().T
        xb = [int(x2[i, 0]) & 1, (int(x2[i, 0]) >> 1) & 1]
        zb = [int(z2[i, 0]) & 1, (int(z2[i, 0]) >> 1) & 1]
        got = _row_matrix(xb, zb, int(r2[i]))
        assert np.allclose(want, got), (C.KIND_NAMES[kind], (x0, z0, x1, z1, s))
        assert int(x2[i, 0]) >> 2 == 0 and int(z2[i, 0]) >> 2 == 0


# ---------------------------------------------------------------- statevector

def _streams(c, seed, shot=0):
    return (S.coin_words(seed, [shot], c.coin_words)[0],
            S.noise_words(seed, [shot], c.noise_words)[0])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7])
def test_oracle_matches_statevector(n):
    """Records equal the brute-force statevector's for the same coins and
    noise draws; random/deterministic agreement is forced by using two
    different coin streams per circuit."""
    for seed in range(40 if n <= 4 else 15):
        circ = C.random_small_circuit(n, 40, seed=seed + 100 * n)
        for cs in (seed, seed + 1000):
            coins, noise = _streams(circ, cs)
            rec = oracle.run(circ, coins, noise)
            bits = oracle.record_bits(rec, circ.n_meas).tolist()
            sv_bits, _ = SV.run(circ, coins, noise)
            assert bits == sv_bits, (n, seed, cs)


def test_random_outcomes_have_probability_half():
    """Every measurement the statevector finds random has p = 1/2 exactly,
    deterministic ones p in {0, 1} (asserted inside SV.measure); and the
    oracle's record follows the coin exactly for the random ones."""
    circ = C.random_small_circuit(6, 60, seed=5, noise=False)
    coins0 = np.zeros(circ.coin_words, np.uint64)
    coins1 = np.full(circ.coin_words, np.uint64(2 ** 64 - 1))
    r0 = oracle.record_bits(oracle.run(circ, coins0), circ.n_meas)
    r1 = oracle.record_bits(oracle.run(circ, coins1), circ.n_meas)
    _, rnd = SV.run(circ, coins0, np.zeros(1, np.uint32))
    m_flags = [r for (k, r) in rnd if int(circ.ops[k]["kind"]) == C.M]
    assert len(m_flags) == circ.n_meas
    # the first random M follows its coin; before it, records agree
    first = next((i for i, f in enumerate(m_flags) if f), None)
    if first is not None:
        assert (r0[:first] == r1[:first]).all()
        assert r0[first] == 0 and r1[first] == 1


# ---------------------------------------------------------------- invariants

def _symplectic_ok(x, z, n):
    W = x.shape[1]
    xb = np.unpackbits(x.view(np.uint8).reshape(2 * n, 8 * W), axis=1, bitorder="little")[:, :n].astype(np.int64)
    zb = np.unpackbits(z.view(np.uint8).reshape(2 * n, 8 * W), axis=1, bitorder="little")[:, :n].astype(np.int64)
    inner = (xb @ zb.T + zb @ xb.T) % 2
    J = np.zeros((2 * n, 2 * n), np.int64)
    J[np.arange(n), np.arange(n) + n] = 1
    J[np.arange(n) + n, np.arange(n)] = 1
    return np.array_equal(inner, J)


def test_invariants_after_every_op():
    """D_i anticommutes with S_i only; all other pairs commute (this also
    implies the 2n rows are independent) -- after every single op."""
    for seed in range(6):
        n = 9
        circ = C.random_small_circuit(n, 80, seed=seed)
        coins, noise = _streams(circ, seed)
        t = oracle.Tableau(n)
        ci = li = 0
        for k in range(len(circ.ops)):
            one = C.Circuit(n, circ.ops[k:k + 1], circ.params)
            kind = int(circ.ops[k]["kind"])
            c1 = np.array([(int(coins[ci >> 6]) >> (ci & 63)) & 1], np.uint64)
            nw = 3 if kind == C.RESET_ERR else 1
            n1 = np.array(noise[li:li + nw] if kind in C.NOISE_KINDS else [0], np.uint32)
            t.run(one, c1, n1)
            ci += kind in (C.M, C.R)
            li += nw if kind in C.NOISE_KINDS else 0
            x, z, _ = t.get()
            assert _symplectic_ok(x, z, n), (seed, k, C.KIND_NAMES[kind])


# ---------------------------------------------------------------- closed forms

def test_ghz_outcomes_equal_first_coin():
    for n in (2, 5, 33, 70):
        c = C.ghz(n)
        for coin in (0, 1):
            rec = oracle.run(c, np.array([coin], np.uint64) if c.coin_words == 1 else
                             np.array([coin] + [0] * (c.coin_words - 1), np.uint64))
            bits = oracle.record_bits(rec, n)
            assert (bits == coin).all()


def test_single_qubit_closed_forms():
    b = C.Builder(3)
    b.measure(0)                     # |0> -> 0 deterministic
    b.gate1(C.X, 1).measure(1)       # X|0> -> 1
    b.gate1(C.H, 2).measure(2)       # |+> -> coin
    b.reset(1).measure(1)            # reset -> 0
    b.gate1(C.H, 0).gate1(C.S, 0).gate1(C.S, 0).gate1(C.H, 0).measure(0)  # HSSH = X
    c = b.build()
    for coins in (0b000000, 0b111111):
        bits = oracle.record_bits(oracle.run(c, np.array([coins], np.uint64)), c.n_meas)
        assert bits.tolist() == [0, 1, coins & 1, 0, 1]


def test_gate_identities_on_tableau():
    """S^4 = I, H^2 = I, CX^2 = I leave the tableau bit-identical."""
    circ = C.random_small_circuit(5, 30, seed=3, noise=False, allow=(C.H, C.S, C.CX, C.CZ))
    t = oracle.Tableau(5)
    t.run(circ)
    ref = t.get()
    b = C.Builder(5)
    for _ in range(4):
        b.gate1(C.S, 2)
    b.gate1(C.H, 1).gate1(C.H, 1).gate2(C.CX, 3, 4).gate2(C.CX, 3, 4)
    t.run(b.build())
    for u, v in zip(ref, t.get()):
        assert np.array_equal(u, v)


# ---------------------------------------------------------------- surface code

@pytest.mark.parametrize("d,rounds", [(3, 1), (3, 3), (5, 2), (5, 5), (7, 7)])
def test_surface_code_noiseless_detectors_zero(d, rounds):
    c = C.surface_code_memory(d, rounds)
    for seed in (0, 1):
        coins, noise = _streams(c, seed)
        bits = oracle.record_bits(oracle.run(c, coins, noise), c.n_meas)
        for det in c.meta["detectors"]:
            assert int(np.bitwise_xor.reduce(bits[det])) == 0
        assert int(np.bitwise_xor.reduce(bits[c.meta["observable"]])) == 0


def test_surface_code_counts():
    for d in (3, 5, 11):
        c = C.surface_code_memory(d)
        cnt = c.counts()
        assert c.n == 2 * d * d - 1
        assert cnt["CX"] == 4 * d * (d - 1) * d
        assert cnt["H"] == (d * d - 1) * d
        assert cnt["M"] == (d * d - 1) * d + d * d
        assert len(c.meta["layout"].x_anc) == len(c.meta["layout"].z_anc) == (d * d - 1) // 2


def test_noisy_surface_code_flags_errors():
    c = C.surface_code_memory(5, p=0.02)
    coins, noise = _streams(c, 3)
    bits = oracle.record_bits(oracle.run(c, coins, noise), c.n_meas)
    nz = sum(int(np.bitwise_xor.reduce(bits[det])) for det in c.meta["detectors"])
    assert nz > 0


# ---------------------------------------------------------------- noise draws

@pytest.mark.parametrize("p", [0.0, 1e-9, 1e-3, 1 / 3, 0.5, 0.999999, 1.0])
def test_threshold_is_exact_floor(p):
    want = min(int(Fraction(p) * 2 ** 32), 2 ** 32)
    assert SV.threshold(p) == want


def test_noise_draw_boundaries():
    """An X error before M flips the outcome; the event test is u < T."""
    for p in (1e-3, 0.3):
        T = SV.threshold(p)
        b = C.Builder(1)
        b.pauli_channel1(0, p, 0.0, 0.0).measure(0)
        c = b.build()
        for u, want in ((0, 1), (T - 1, 1), (T, 0), (2 ** 32 - 1, 0)):
            bits = oracle.record_bits(oracle.run(c, np.zeros(1, np.uint64),
                                                 np.array([u], np.uint32)), 1)
            assert int(bits[0]) == want, (p, u)


def test_depolarize_index_nearly_uniform():
    T = SV.threshold(1e-3)
    for K in (3, 15):
        counts = np.bincount([(u * K) // T for u in range(0, T, 997)], minlength=K)
        assert counts.max() - counts.min() <= 2 + counts.max() // 1000


# ---------------------------------------------------------------- errors

def test_oracle_rejects_bad_input():
    b = C.Builder(2)
    b.gate2(C.CX, 0, 0)
    with pytest.raises(oracle.OracleError):
        oracle.run(b.build())
    b = C.Builder(2)
    b.gate1(C.H, 5)
    with pytest.raises(oracle.OracleError):
        oracle.run(b.build())
    b = C.Builder(2)
    for _ in range(70):
        b.measure(0)
    c = b.build()
    with pytest.raises(oracle.OracleError):
        t = oracle.Tableau(2)
        t.run(c, np.zeros(1, np.uint64))     # 70 coin slots need 2 words


def test_sample_threads_match_single():
    c = C.surface_code_memory(3, p=0.05)
    coins, noise = S.streams_for(c, 0, range(64))
    r1, _ = oracle.sample(c, coins, noise, threads=1)
    r4, _ = oracle.sample(c, coins, noise, threads=4)
    assert np.array_equal(r1, r4)
    for s in (0, 17, 63):
        assert np.array_equal(r1[s], oracle.run(c, coins[s], noise[s]))


# ---------------------------------------------------------------- generators

def test_splitmix64_published_first_output():
    # SplitMix64 with state 0: first output 0xE220A8397B1DCDAF
    assert int(S.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    assert int(S.splitmix64(0, 2)[1]) == S.mix64_int(2 * S.GAMMA)


def test_streams_are_keyed_by_shot():
    a = S.coin_words(0, [0, 1, 2], 4)
    b = S.coin_words(0, [2], 4)
    assert np.array_equal(a[2], b[0])
    assert not np.array_equal(a[0], a[1])


def test_random_measurement_moves_pivot_row_to_destabilizer():
    """Sec. 2.4: after a random measurement the old pivot stabilizer (sign
    included) is stored in its destabilizer and the pivot becomes +-Z_a.
    Worked by hand: H then Z on |0> gives D=Z, S=-X; measuring gives D=-X,
    S=(-1)^coin Z."""
    b = C.Builder(1)
    b.gate1(C.H, 0).gate1(C.Z, 0).measure(0)
    c = b.build()
    for coin in (0, 1):
        t = oracle.Tableau(1)
        t.run(c, np.array([coin], np.uint64))
        x, z, r = t.get()
        assert (int(x[0, 0]), int(z[0, 0]), int(r[0])) == (1, 0, 1)
        assert (int(x[1, 0]), int(z[1, 0]), int(r[1])) == (0, 1, coin)


def test_serving_trace_is_seeded_poisson():
    from paper_2507_03092_gb300 import serve_trace as T
    a = T.make_trace(200.0, 60.0, seed=0)
    b = T.make_trace(200.0, 60.0, seed=0)
    assert [(r.t_arrival, r.d, r.shots) for r in a] == [(r.t_arrival, r.d, r.shots) for r in b]
    assert 11000 < len(a) < 13000                       # ~ rate * duration
    gaps = np.diff([r.t_arrival for r in a])
    assert abs(gaps.mean() - 1 / 200.0) < 2e-4
    assert {r.d for r in a} == set(range(3, 32, 2))
    shots = np.array([r.shots for r in a])
    assert shots.min() >= 1 and shots.max() <= 256 and abs(shots.mean() - 128.5) < 5
    assert len({r.seed for r in a}) == len(a)            # streams keyed per request


def test_composite_t1t2_mixture_equals_kraus_composition():
    """Sec. 4.2: reset w.p. gamma then Z w.p. q (the RESET_ERROR channel with
    composite_t1t2_probs) equals dephasing after amplitude damping, for random
    states and T1 >= T2."""
    rng = np.random.default_rng(3)
    Zm = np.diag([1.0, -1.0]).astype(complex)
    P0 = np.diag([1.0, 0.0]).astype(complex)
    for _ in range(200):
        T1 = float(rng.uniform(20, 200))
        T2 = float(rng.uniform(5, T1))
        t = float(rng.uniform(0, 3 * T1))
        a = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
        rho = a @ a.conj().T
        rho /= np.trace(rho)
        g = 1 - np.exp(-t / T1)                         # amplitude damping
        K0 = np.array([[1, 0], [0, np.sqrt(1 - g)]], complex)
        K1 = np.array([[0, np.sqrt(g)], [0, 0]], complex)
        ad = K0 @ rho @ K0.conj().T + K1 @ rho @ K1.conj().T
        pd = (1 - np.exp(-t * (1 / T2 - 1 / (2 * T1)))) / 2   # extra dephasing to reach T2
        want = (1 - pd) * ad + pd * Zm @ ad @ Zm
        gamma, q = C.composite_t1t2_probs(T1, T2, t)
        reset = np.trace(rho) * P0
        mix = (1 - gamma) * rho + gamma * reset
        got = (1 - q) * mix + q * Zm @ mix @ Zm
        assert np.allclose(got, want, atol=1e-12)
    with pytest.raises(ValueError):
        C.composite_t1t2_probs(50.0, 60.0, 1.0)


# ---------------------------------------------------------------- Pauli products

def _pauli_kron(xbits, zbits):
    m = np.eye(1, dtype=complex)
    for xb, zb in zip(xbits, zbits):
        m = np.kron(pauli_matrix((int(xb), int(zb))), m)     # qubit 0 least significant
    return m


def _bits(words, n):
    w = np.ascontiguousarray(words, np.uint64)
    return np.unpackbits(w.view(np.uint8), bitorder="little")[:n]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_commute_matches_matrix_commutation(n):
    """Sec. 3.2's commutation equation, checked against P S = -S P for the
    dense 2^n x 2^n matrices of every tableau row and random Paulis."""
    rng = np.random.default_rng(n)
    for seed in range(6):
        circ = C.random_small_circuit(n, 30, seed=seed + 10 * n, noise=False)
        coins, noise = _streams(circ, seed)
        t = oracle.Tableau(n)
        t.run(circ, coins, noise)
        x, z, _ = t.get()
        px = rng.integers(0, 2 ** n, size=(8, 1), dtype=np.uint64)
        pz = rng.integers(0, 2 ** n, size=(8, 1), dtype=np.uint64)
        got = t.commute(px, pz)
        for k in range(8):
            P = _pauli_kron(_bits(px[k], n), _bits(pz[k], n))
            for i in range(2 * n):
                Srow = _pauli_kron(_bits(x[i], n), _bits(z[i], n))
                anti = not np.allclose(P @ Srow, Srow @ P)
                assert anti == bool((int(got[k, i // 64]) >> (i % 64)) & 1), (seed, k, i)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_mpp_matches_statevector(n):
    """Pauli-product measurements interleaved with gates, M, R and noise:
    records equal the statevector's projective measurement of P."""
    for seed in range(25 if n <= 3 else 10):
        circ = C.random_small_circuit(n, 40, seed=seed + 500 * n, mpp=True)
        assert int(np.count_nonzero(circ.ops["kind"] == C.MPP)) > 0
        for cs in (seed, seed + 1000):
            coins, noise = _streams(circ, cs)
            bits = oracle.record_bits(oracle.run(circ, coins, noise), circ.n_meas).tolist()
            sv_bits, _ = SV.run(circ, coins, noise)
            assert bits == sv_bits, (n, seed, cs)


def test_mpp_of_single_z_is_m():
    """MPP of one Z factor is the Z measurement: same records and the same
    tableau, row for row."""
    for seed in range(5):
        circ = C.random_small_circuit(6, 60, seed=seed)
        b = C.Builder(6)
        for o in circ.ops:
            if int(o["kind"]) == C.M:
                b.mpp([(int(o["q0"]), "Z")])
            else:
                b.op(int(o["kind"]), int(o["q0"]), int(o["q1"]), int(o["arg"]))
        alt = b.build()
        alt.params = circ.params
        coins, noise = _streams(circ, seed)
        r1, t1, _ = oracle.run(circ, coins, noise, return_tableau=True)
        r2, t2, _ = oracle.run(alt, coins, noise, return_tableau=True)
        assert np.array_equal(r1, r2)
        for a, b_ in zip(t1, t2):
            assert np.array_equal(a, b_)


def test_mpp_ghz_closed_forms():
    """GHZ_3 = (|000> + |111>)/sqrt2: XXX = +1, XYY = YXY = YYX = -1,
    Z0 Z1 = Z1 Z2 = +1 -- deterministic whatever the coins."""
    for coin in (0, 1):
        b = C.Builder(3)
        b.gate1(C.H, 0)
        b.gate2(C.CX, 0, 1)
        b.gate2(C.CX, 1, 2)
        for f in ("XXX", "XYY", "YXY", "YYX"):
            b.mpp([(q, ch) for q, ch in enumerate(f)])
        b.mpp([(0, "Z"), (1, "Z")])
        b.mpp([(2, "Z"), (1, "Z")])
        c = b.build()
        t = oracle.Tableau(3)
        bits = oracle.record_bits(t.run(c, np.array([2 ** 64 - 1 if coin else 0], np.uint64)), 6)
        assert bits.tolist() == [0, 1, 1, 1, 0, 0]
        assert t.stats.n_meas_random == 0 and t.stats.n_meas_det == 6


def test_mpp_random_outcome_installs_signed_product():
    """A random MPP outcome c leaves (-1)^c P in the stabilizer group:
    measuring P again is deterministic with the same outcome, and Z-basis
    products that commute with P keep their values."""
    b = C.Builder(4)
    b.mpp([(0, "X"), (1, "Y"), (3, "Z")])
    b.mpp([(0, "X"), (1, "Y"), (3, "Z")])
    b.mpp([(2, "Z")])
    c = b.build()
    for coin in (0, 1):
        t = oracle.Tableau(4)
        bits = oracle.record_bits(t.run(c, np.array([coin], np.uint64)), 3)
        assert bits.tolist() == [coin, coin, 0]
        assert t.stats.n_meas_random == 1


def test_mpp_rejects_bad_factor_lists():
    for ops in ([(C.MPP, 2, 0), (C.PAULI, 0, 3)],                     # too few factors
                [(C.MPP, 2, 0), (C.PAULI, 0, 3), (C.PAULI, 0, 1)],   # repeated qubit
                [(C.MPP, 1, 0), (C.PAULI, 0, 4)],                    # bad Pauli code
                [(C.MPP, 1, 0), (C.H, 0, 0)],                        # factor is not PAULI
                [(C.MPP, 0, 0)]):                                    # no factors
        b = C.Builder(2)
        for k, q0, q1 in ops:
            b.op(k, q0, q1)
        with pytest.raises(oracle.OracleError):
            oracle.run(b.build(), np.zeros(1, np.uint64))


def test_invariants_after_every_mpp():
    """The symplectic invariants hold after every Pauli-product measurement
    (each MPP with its factors run as one unit)."""
    for seed in range(6):
        n = 8
        circ = C.random_small_circuit(n, 60, seed=seed + 77, noise=False, mpp=True)
        coins, _ = _streams(circ, seed)
        t = oracle.Tableau(n)
        ci, k, ops = 0, 0, circ.ops
        while k < len(ops):
            kind = int(ops[k]["kind"])
            w = 1 + (int(ops[k]["q0"]) if kind == C.MPP else 0)
            c1 = np.array([(int(coins[ci >> 6]) >> (ci & 63)) & 1], np.uint64)
            t.run(C.Circuit(n, ops[k:k + w], circ.params), c1, np.zeros(1, np.uint32))
            ci += kind in (C.M, C.R, C.MPP)
            k += w
            x, z, _ = t.get()
            assert _symplectic_ok(x, z, n), (seed, k)


@pytest.mark.parametrize("d", [3, 5])
def test_mpp_surface_code_noiseless_detectors_zero(d):
    """Checks measured as Pauli products: every detector is 0 without noise
    (whatever the coins); later rounds are deterministic."""
    c = C.surface_code_mpp(d, rounds=3)
    for seed in (0, 1, 2):
        coins, noise = _streams(c, seed)
        t = oracle.Tableau(c.n)
        bits = oracle.record_bits(t.run(c, coins, noise), c.n_meas)
        for det in c.meta["detectors"]:
            assert int(np.bitwise_xor.reduce(bits[det])) == 0
        assert int(np.bitwise_xor.reduce(bits[c.meta["observable"]])) == 0
        n_x = sum(1 for pl in C.surface_layout(d).plaquettes if pl[2] == "X")
        n_z = sum(1 for pl in C.surface_layout(d).plaquettes if pl[2] == "Z")
        # random: the round-1 X checks, and the final data measurements beyond
        # what the Z checks and the logical Z fix
        assert t.stats.n_meas_random == n_x + (d * d - n_z - 1)


def test_mpp_surface_code_flags_errors():
    c = C.surface_code_mpp(5, rounds=5, p=0.02)
    fired = 0
    for seed in range(8):
        coins, noise = _streams(c, seed)
        bits = oracle.record_bits(oracle.run(c, coins, noise), c.n_meas)
        fired += sum(int(np.bitwise_xor.reduce(bits[det])) for det in c.meta["detectors"])
    assert fired > 0


# ---------------------------------------------------------------- reorderings the GPU path relies on
# The layered engine applies a layer's Z measurements out of circuit order:
# random ones in waves of pairwise-commuting ops, deterministic ones from the
# layer's starting state, Pauli errors (and the X after a reset) at the end of
# the layer.  Each rule is checked here on the oracle alone, bit for bit.

def _rows_bits(words, n):
    return np.unpackbits(words.view(np.uint8).reshape(words.shape[0], -1), axis=1,
                         bitorder="little")[:, :n].astype(bool)


def _random_state(n, seed, n_gates=80):
    """Tableau after a seeded random H/S/CX circuit from |0...0>."""
    rng = np.random.default_rng(seed)
    b = C.Builder(n)
    for _ in range(n_gates):
        k = int(rng.integers(3))
        if k == 2:
            a, c = (int(v) for v in rng.choice(n, size=2, replace=False))
            b.gate2(C.CX, a, c)
        else:
            b.gate1(C.H if k == 0 else C.S, int(rng.integers(n)))
    t = oracle.Tableau(n)
    t.run(b.build())
    return t.get()


def _run_from(state, n, build, coin_bits):
    """Apply the ops added by ``build(builder)`` to a copy of ``state``; coin k
    goes to the k-th M.  Returns (record bits, tableau)."""
    b = C.Builder(n)
    build(b)
    circ = b.build()
    coins = np.zeros(max(1, circ.coin_words), np.uint64)
    for k, c in enumerate(coin_bits):
        coins[k >> 6] |= np.uint64(int(c) << (k & 63))
    t = oracle.Tableau(n)
    t.set(*state)
    rec = t.run(circ, coins)
    return oracle.record_bits(rec, circ.n_meas), t.get()


def _pivot(xb, n, a):
    """First stabilizer row with an X or Y on qubit a (Sec. 2.4), or None."""
    s = np.nonzero(xb[n:, a])[0]
    return None if len(s) == 0 else n + int(s[0])


def _same_tableau(t1, t2):
    return all(np.array_equal(u, v) for u, v in zip(t1, t2))


def test_commuting_random_measurements_reorder_bit_for_bit():
    """Two random Z measurements whose pivot rows have no X or Y on each
    other's qubit leave the same tableau (x, z and every sign) and the same
    outcomes in either order, for every pair of coins; this is the rule that
    lets random measurements run in waves.  Pairs that break the condition
    are not covered by it, and some of them do differ (so the test can
    fail)."""
    n = 18
    n_cond = n_diff = 0
    for seed in range(10):
        state = _random_state(n, seed)
        xb = _rows_bits(state[0], n)
        for a, b in itertools.permutations(range(n), 2):
            pa, pb = _pivot(xb, n, a), _pivot(xb, n, b)
            if pa is None or pb is None or a > b:
                continue
            cond = not xb[pa, b] and not xb[pb, a]
            for ca, cb in itertools.product((0, 1), repeat=2):
                r1, t1 = _run_from(state, n, lambda B: B.measure(a).measure(b), (ca, cb))
                r2, t2 = _run_from(state, n, lambda B: B.measure(b).measure(a), (cb, ca))
                same = _same_tableau(t1, t2) and r1[0] == r2[1] and r1[1] == r2[0]
                if cond:
                    assert same, (seed, a, b, ca, cb)
                    assert (r1[0], r1[1]) == (ca, cb)      # both stay random
                elif not same:
                    n_diff += 1
            n_cond += cond
    assert n_cond >= 50 and n_diff > 0, (n_cond, n_diff)


def test_deterministic_outcomes_fixed_by_the_layer_start():
    """A Z measurement that is deterministic when its layer starts has the
    outcome it has when measured alone at the layer start, whatever the
    layer's other Z measurements (random or not, any coins) do first; this is
    why all deterministic ops of a layer are resolved from its starting
    state."""
    n = 16
    checked = 0
    rng = np.random.default_rng(3)
    for seed in range(12):
        state = _random_state(n, 100 + seed, n_gates=50)
        xb = _rows_bits(state[0], n)
        det = [a for a in range(n) if _pivot(xb, n, a) is None]
        alone = {a: int(_run_from(state, n, lambda B, a=a: B.measure(a), (0,))[0][0]) for a in det}
        for _ in range(6):
            order = [int(q) for q in rng.permutation(n)]
            coins = rng.integers(0, 2, size=n)
            bits, _ = _run_from(state, n, lambda B: [B.measure(q) for q in order], coins)
            for k, q in enumerate(order):
                if q in alone:
                    assert int(bits[k]) == alone[q], (seed, q, order)
                    checked += 1
    assert checked > 100


@pytest.mark.parametrize("pauli", [C.X, C.Y, C.Z])
def test_pauli_on_another_qubit_commutes_with_measurement(pauli):
    """A Pauli on qubit c (a noise error, or the X that finishes a reset)
    and a Z measurement of qubit a != c give the same tableau, bit for bit,
    and the same outcome in either order; this is why the layered engine
    applies a layer's Pauli errors and reset flips after its measurements."""
    n = 12
    for seed in range(8):
        state = _random_state(n, 200 + seed, n_gates=40)
        for a in range(n):
            for c in range(n):
                if a == c:
                    continue
                for coin in (0, 1):
                    r1, t1 = _run_from(state, n, lambda B: B.gate1(pauli, c).measure(a), (coin,))
                    r2, t2 = _run_from(state, n, lambda B: B.measure(a).gate1(pauli, c), (coin,))
                    assert r1[0] == r2[0] and _same_tableau(t1, t2), (seed, a, c, coin)


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_reset_error_matches_statevector(n):
    """RESET_ERROR (reset with the second draw's coin when the first is below
    T(gamma), then Z when the third is below T(q)) inside random circuits:
    records equal the statevector's for the same draws.  gamma = q = 1/2
    makes every branch frequent, and H before some final measurements makes
    the Z errors visible."""
    rng = np.random.default_rng(70 + n)
    for seed in range(12):
        b = C.Builder(n)
        for _ in range(40):
            k = int(rng.integers(6))
            q = int(rng.integers(n))
            if k == 0:
                b.gate1(C.H, q)
            elif k == 1:
                b.gate1(C.S, q)
            elif k == 2 and n > 1:
                b.gate2(C.CX, q, (q + 1 + int(rng.integers(n - 1))) % n)
            elif k == 3:
                b.measure(q)
            else:
                b.reset_error(q, 0.5, 0.5)
        for q in range(n):
            if rng.integers(2):
                b.gate1(C.H, q)
            b.measure(q)
        circ = b.build()
        for cs in (seed, seed + 500):
            coins, noise = _streams(circ, cs)
            bits = oracle.record_bits(oracle.run(circ, coins, noise), circ.n_meas).tolist()
            sv_bits, _ = SV.run(circ, coins, noise)
            assert bits == sv_bits, (n, seed, cs)
