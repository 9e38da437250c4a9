"""The layered engine replays its launch sequence as a CUDA graph when
per-launch profiling is off.  Graph replay must give the records (and the
tableau) of plain launches: over repeated calls (executable graphs updated in
place), changing shot counts (new graph topology), circuits with Pauli-product
measurements, and interleaved with other work on the caller's stream."""
import numpy as np
import pytest

import oracle
from paper_2507_03092_gb300 import binding as B
from paper_2507_03092_gb300 import circuit as C
from paper_2507_03092_gb300 import streams as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = B.Simulator(0)
    yield s
    s.close()


def _run(sim, cid, circ, coins, noise, profiled):
    B.stab_profile(sim.ctx, 0xFF if profiled else 0)
    try:
        out = B.records_to_numpy(sim.sample(cid, circ, coins.shape[0], coins, noise, engine=B.ENGINE_LAYERED))
        sim.sync()
    finally:
        B.stab_profile(sim.ctx, 0)
    return out


@pytest.mark.parametrize("kind", ["surface", "random", "mpp"])
def test_graph_replay_equals_plain_launches(sim, kind):
    if kind == "surface":
        circ = C.surface_code_memory(9, p=5e-3)
    elif kind == "random":
        circ = C.random_clifford_layers(300, 40, seed=3)
    else:
        circ = C.random_small_circuit(70, 400, seed=4, mpp=True)
    cid = sim.compile(circ)
    for rep, shots in enumerate((5, 5, 5, 2, 7, 7)):
        coins, noise = S.streams_for(circ, 40 + rep, range(shots))
        g = _run(sim, cid, circ, coins, noise, profiled=False)
        p = _run(sim, cid, circ, coins, noise, profiled=True)
        assert np.array_equal(g, p), (kind, rep)
        if rep in (0, 3):
            want, _ = oracle.sample(circ, coins, noise)
            assert np.array_equal(g, want), (kind, rep)


def test_graph_replay_orders_with_caller_stream(sim):
    """Work queued on the caller's stream before and after a replayed call
    sees the call's results in order (records copied right after the call)."""
    torch = pytest.importorskip("torch")
    circ = C.surface_code_memory(5, p=1e-2)
    cid = sim.compile(circ)
    coins, noise = S.streams_for(circ, 9, range(16))
    want, _ = oracle.sample(circ, coins, noise)
    dc, dn = sim.to_dev(coins), sim.to_dev(noise)
    for _ in range(3):
        rec = sim.record_buffer(16, circ.record_words)
        rec.fill_(-1)                                 # queued before the call
        B.stab_sample(sim.ctx, cid, 16, B.make_streams(B.STREAM_BUFFER, coins=dc, noise=dn), rec,
                      B.ENGINE_LAYERED)
        copy = rec.clone()                            # queued after the call
        torch.cuda.synchronize()
        assert np.array_equal(B.records_to_numpy(copy), want)


def test_apply_circuit_graph_replay_tableau(sim):
    circ = C.random_small_circuit(40, 200, seed=8)
    coins, noise = S.streams_for(circ, 2, [0])
    want, wtab, _ = oracle.run(circ, coins[0], noise[0], return_tableau=True)
    cid = sim.compile(circ)
    for _ in range(2):
        B.stab_tableau_init(sim.ctx, circ.n, 1)
        rec = sim.record_buffer(1, circ.record_words)
        B.stab_apply_circuit(sim.ctx, cid, B.make_streams(B.STREAM_BUFFER, coins=sim.to_dev(coins),
                                                          noise=sim.to_dev(noise)), rec)
        sim.sync()
        assert np.array_equal(B.records_to_numpy(rec)[0], want)
        for g, w in zip(B.stab_get_tableau(sim.ctx, 0, circ.n), wtab):
            assert np.array_equal(g, w)


def test_long_program_runs_without_one_graph():
    """A launch sequence longer than the graph budget (here the random n-wide
    benchmark at n = 48 with 1200 rounds: several thousand layers) is issued
    as plain launches instead of one captured graph; its records still match
    the oracle's, over two calls."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    circ = C.random_wide_benchmark(48, 1200, seed=7)
    s = B.Simulator(0)
    try:
        cid = s.compile(circ)
        assert s.info(cid)["n_layers"] > 2000
        coins, noise = S.streams_for(circ, 5, range(2))
        want, _ = oracle.sample(circ, coins, noise)
        for _ in range(2):
            got = B.records_to_numpy(s.sample(cid, circ, 2, coins, noise, engine=B.ENGINE_LAYERED))
            s.sync()
            assert np.array_equal(got, want)
    finally:
        s.close()


def test_graph_replay_across_wave_cluster_sizes(sim):
    """The wave kernel's cluster size (CTAs per tableau) follows the batch
    size: 8 for a few tableaux, fewer for larger batches, 1 from 77 on.  It
    is a launch attribute of the captured graph, so one circuit sampled with
    batch sizes that change it must still give the oracle's records each
    time (the executable graph is instantiated anew, not updated in place)."""
    circ = C.surface_code_memory(5, p=5e-3)
    cid = sim.compile(circ)
    for shots in (1, 20, 3, 40, 1, 77, 2, 20):
        coins, noise = S.streams_for(circ, 100 + shots, range(shots))
        got = _run(sim, cid, circ, coins, noise, profiled=False)
        want, _ = oracle.sample(circ, coins, noise)
        assert np.array_equal(got, want), shots


def test_graph_replay_many_measurement_layers(sim):
    """A one-tableau program of 21 measurement layers (a d = 5 memory circuit
    with 20 syndrome rounds), noiseless (later rounds have deterministic
    outcomes only) and noisy: graph replay gives the records of plain
    launches and of the oracle, with the same number of kernel launches
    (after a first run that finds the layers without random outcomes)."""
    for p in (0.0, 5e-3):
        circ = C.surface_code_memory(5, rounds=20, p=p)
        cid = sim.compile(circ)
        coins, noise = S.streams_for(circ, 17, [0])
        _run(sim, cid, circ, coins, noise, profiled=False)
        B.stab_launch_count(sim.ctx, reset=True)
        plain = _run(sim, cid, circ, coins, noise, profiled=True)
        n_plain = B.stab_launch_count(sim.ctx, reset=True)
        for _ in range(3):
            graph = _run(sim, cid, circ, coins, noise, profiled=False)
            n_graph = B.stab_launch_count(sim.ctx, reset=True)
            assert np.array_equal(graph, plain), p
            assert n_graph == n_plain, (n_plain, n_graph)
        want, _ = oracle.sample(circ, coins, noise)
        assert np.array_equal(plain, want), p


def test_deterministic_layers_leave_out_random_kernels(sim):
    """Which Z measurements are random is fixed by the circuit from |0...0>
    (Pauli noise, outcomes and reset corrections change signs only): after
    the first run of a program the engine leaves out the random-measurement
    launches of the layers that had no random op, and every run, before and
    after, gives the oracle's records on fresh streams.  A circuit with
    RESET_ERROR (a reset drawn by noise) keeps every launch."""
    circ = C.surface_code_memory(5, rounds=20, p=5e-3)
    cid = sim.compile(circ)
    counts = []
    for rep in range(4):
        coins, noise = S.streams_for(circ, 300 + rep, range(3))
        B.stab_launch_count(sim.ctx, reset=True)
        got = _run(sim, cid, circ, coins, noise, profiled=rep == 3)
        counts.append(B.stab_launch_count(sim.ctx, reset=True))
        want, _ = oracle.sample(circ, coins, noise)
        assert np.array_equal(got, want), rep
    # two measurement layers have random ops (the first round's, whose X-type
    # ancillas are random, and the final data layer): every other one runs
    # 3 launches fewer
    n_ml = sim.info(cid)["n_meas_layers"]
    assert counts[0] - counts[1] == (n_ml - 2) * 3, (counts, n_ml)
    assert counts[1] == counts[2] == counts[3], counts

    # a qubit in |+> then RESET_ERROR: its measurement is random or not by the
    # reset's own draw, so no layer may be left out
    b = C.Builder(6)
    rng = np.random.default_rng(1)
    for _ in range(30):
        for q in range(6):
            b.gate1(C.H, q)
        for q in range(6):
            b.reset_error(q, 0.5, 0.1)
        for q in range(0, 6, 2):
            b.gate2(C.CX, q, q + 1)
        for q in range(6):
            if rng.integers(2):
                b.measure(q)
    circ = b.build()
    cid = sim.compile(circ)
    counts = []
    for rep in range(3):
        coins, noise = S.streams_for(circ, 400 + rep, range(3))
        B.stab_launch_count(sim.ctx, reset=True)
        got = _run(sim, cid, circ, coins, noise, profiled=False)
        counts.append(B.stab_launch_count(sim.ctx, reset=True))
        want, _ = oracle.sample(circ, coins, noise)
        assert np.array_equal(got, want), rep
    assert counts[0] == counts[1] == counts[2], counts
