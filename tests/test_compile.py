"""Host logic of the circuit compiler (validation, layering, stream sizes)
through stab_compile_info, which compiles without a context or a GPU."""
import numpy as np
import pytest

from paper_2507_03092_gb300 import binding as B
from paper_2507_03092_gb300 import build as BLD
from paper_2507_03092_gb300 import circuit as C


@pytest.fixture(scope="module", autouse=True)
def _lib():
    BLD.build()


def info(circ):
    return B.stab_compile_info(circ)


def _ops(n, ops, params=()):
    b = C.Builder(n)
    for p in params:
        b._param(p)
    for o in ops:
        b.op(*o)
    return b.build()


# ---------------------------------------------------------------- sizes

def _circuits():
    yield C.surface_code_memory(3)
    for d, p in ((3, 1e-3), (5, 2e-2), (9, 1e-3)):
        yield C.surface_code_memory(d, p=p)
    yield C.surface_code_mpp(5, p=1e-2)
    yield C.random_clifford_layers(200, 30, seed=4)
    yield C.random_wide_benchmark(64, seed=2)
    for s in range(6):
        yield C.random_small_circuit(9 + 13 * s, 300, seed=s, mpp=s % 2 == 1)


def test_sizes_match_the_python_circuit_model():
    """Record bits, coin slots and noise draws the compiler reports equal the
    counts the Python circuit model takes from the op list itself (an
    independent count: one record bit per M or MPP, one coin per M, R or MPP,
    one draw per noise op and three per RESET_ERROR)."""
    for circ in _circuits():
        I = info(circ)
        k = circ.ops["kind"]
        assert I["n"] == circ.n
        assert I["n_meas"] == circ.n_meas
        assert I["n_coin"] == circ.n_coin
        assert I["n_noise_words"] == circ.n_noise
        assert I["record_words"] == circ.record_words
        assert I["coin_words"] == circ.coin_words
        assert I["n_gates"] == int(np.count_nonzero(np.isin(k, C.ONE_QUBIT_GATES + C.TWO_QUBIT_GATES)))
        assert I["n_ops"] == int(np.count_nonzero(~np.isin(k, (C.NOP, C.TICK, C.PAULI))))
        assert I["n_layers"] == I["n_gate_layers"] + I["n_meas_layers"]


@pytest.mark.parametrize("d", [3, 5, 7, 11])
def test_surface_code_closed_forms(d):
    """Rotated surface-code Z-memory, d rounds: (d^2 - 1) H and 4d(d - 1) CX
    per round, d^2 - 1 ancilla measurements per round plus d^2 data
    measurements, one reset of every qubit and then of every ancilla between
    rounds; per round one gate run of six layers (H, four CX steps, H); the
    measurement layers are the initial reset, one per round, and the last
    round's ancillas share theirs with the data qubits (disjoint qubits)."""
    circ = C.surface_code_memory(d, p=1e-3)
    I = info(circ)
    n, na = 2 * d * d - 1, d * d - 1
    assert I["n"] == n
    assert I["n_gates"] == d * (na + 4 * d * (d - 1))
    assert I["n_meas"] == d * na + d * d
    assert I["n_coin"] == I["n_meas"] + n + (d - 1) * na
    assert I["n_gate_layers"] == 6 * d
    assert I["n_gate_runs"] == d
    assert I["n_meas_layers"] == d + 1
    assert I["max_layer_meas"] == n


# ---------------------------------------------------------------- layering

H, S, CX, M, R, TICK = C.H, C.S, C.CX, C.M, C.R, C.TICK


@pytest.mark.parametrize("ops,gl,ml,runs,maxm", [
    ([(H, 0), (H, 1), (H, 2)], 1, 0, 1, 0),                    # disjoint gates share a layer
    ([(H, 0), (H, 0)], 2, 0, 1, 0),                            # a qubit twice: two layers, one run
    ([(CX, 0, 1), (CX, 2, 3)], 1, 0, 1, 0),
    ([(CX, 0, 1), (CX, 1, 2)], 2, 0, 1, 0),
    ([(H, 0), (TICK,), (H, 1)], 1, 0, 1, 0),                   # TICK is only a hint
    ([(M, 0), (M, 1)], 0, 1, 0, 2),
    ([(M, 0), (M, 0)], 0, 2, 0, 1),
    ([(M, 0), (R, 0)], 0, 1, 0, 1),                            # R right after M folds into it
    ([(R, 0), (R, 0)], 0, 1, 0, 1),                            # and after R
    ([(H, 0), (M, 1), (H, 0)], 2, 1, 2, 1),                    # measurement between two runs
    ([(H, 0), (H, 1), (M, 0), (M, 1), (H, 0)], 2, 1, 2, 2),
])
def test_layering(ops, gl, ml, runs, maxm):
    I = info(_ops(4, ops))
    assert (I["n_gate_layers"], I["n_meas_layers"], I["n_gate_runs"], I["max_layer_meas"]) == \
        (gl, ml, runs, maxm), ops


def test_folded_reset_keeps_its_coin_slot():
    I = info(_ops(2, [(M, 0), (R, 0), (M, 1)]))
    assert (I["n_meas"], I["n_coin"], I["n_meas_layers"]) == (2, 3, 1)


def test_noise_attaches_to_its_gate():
    """A noise op on the qubits of the gate just before it joins that gate's
    item (no extra layer); on other qubits it is an item of its own."""
    b = C.Builder(3)
    b.gate1(H, 0).dep1(0, 0.1).gate2(CX, 1, 2).dep2(1, 2, 0.1)
    I = info(b.build())
    assert (I["n_gate_layers"], I["n_noise_words"]) == (1, 2)
    b = C.Builder(3)
    b.gate1(H, 0).dep1(0, 0.1).dep1(0, 0.2).dep1(0, 0.3)     # two attach, the third cannot
    I = info(b.build())
    assert (I["n_gate_layers"], I["n_noise_words"]) == (2, 3)


def test_mpp_layers():
    b = C.Builder(3)
    b.mpp([(0, "X"), (1, "Z")]).measure(2)
    assert info(b.build())["n_meas_layers"] == 1
    b = C.Builder(3)
    b.mpp([(0, "X"), (1, "Z")]).measure(1)
    I = info(b.build())
    assert (I["n_meas_layers"], I["n_meas"], I["n_coin"]) == (2, 2, 2)


# ---------------------------------------------------------------- validation

P = C.PAULI


@pytest.mark.parametrize("n,ops,params", [
    (2, [(H, 2)], ()),                                  # qubit out of range
    (2, [(CX, 0, 0)], ()),                              # two-qubit op on one qubit
    (2, [(CX, 0, 2)], ()),
    (2, [(C.DEP1, 0, 0, 1)], [(0.1,)]),                 # parameter row out of range
    (2, [(C.DEP1, 0, 0, 0)], [(-0.1,)]),                # probability outside [0, 1]
    (2, [(C.DEP1, 0, 0, 0)], [(1.5,)]),
    (2, [(C.DEP1, 0, 0, 0)], [(float("nan"),)]),
    (2, [(C.PC1, 0, 0, 0)], [(0.5, 0.4, 0.2)]),         # Pauli channel above 1
    (2, [(99, 0)], ()),                                 # unknown kind
    (2, [(P, 0, 1)], ()),                               # PAULI outside an MPP
    (2, [(C.MPP, 0, 0), (H, 0)], ()),                   # MPP without factors
    (2, [(C.MPP, 2, 0), (P, 0, 1)], ()),                # fewer factors than announced
    (2, [(C.MPP, 2, 0), (P, 0, 1), (P, 0, 3)], ()),     # repeated qubit
    (2, [(C.MPP, 1, 0), (P, 0, 4)], ()),                # factor code outside 1..3
    (2, [(C.MPP, 1, 0), (P, 2, 1)], ()),                # factor qubit out of range
    (2, [(C.MPP, 1, 0), (H, 0)], ()),                   # factor that is not a PAULI
    (70, [(C.MPP, 65, 0)] + [(P, q, 3) for q in range(65)], ()),   # more than 64 factors
])
def test_invalid_circuits_are_rejected(n, ops, params):
    with pytest.raises(B.StabError) as e:
        info(_ops(n, ops, params))
    assert e.value.code == B.ERR_ARG
    assert str(e.value)


def test_zero_qubits_rejected_and_empty_circuit_accepted():
    with pytest.raises(B.StabError) as e:
        info(C.Builder(0).build())
    assert e.value.code == B.ERR_ARG
    I = info(C.Builder(5).build())
    assert (I["n_layers"], I["n_meas"], I["record_words"], I["coin_words"]) == (0, 0, 1, 1)


def test_largest_mpp_accepted():
    b = C.Builder(64)
    b.mpp([(q, "XYZ"[q % 3]) for q in range(64)])
    I = info(b.build())
    assert (I["n_meas"], I["n_meas_layers"]) == (1, 1)
