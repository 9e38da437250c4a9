"""GPU path vs CPU oracle: measurement records (bit-exact) and full tableaux
(x, z and every sign bit, including destabilizer signs), through the C ABI."""
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


def _apply_layered(sim, circ, coins, noise, count=1):
    """Resident tableaux + apply_circuit (layered engine); returns records and
    the tableaux."""
    cid = sim.compile(circ)
    B.stab_tableau_init(sim.ctx, circ.n, count)
    dc, dn = sim.to_dev(coins.reshape(count, -1)), sim.to_dev(noise.reshape(count, -1))
    rec = sim.record_buffer(count, circ.record_words)
    B.stab_apply_circuit(sim.ctx, cid, B.make_streams(B.STREAM_BUFFER, coins=dc, noise=dn), rec)
    sim.sync()
    tabs = [B.stab_get_tableau(sim.ctx, i, circ.n) for i in range(count)]
    B.stab_release_circuit(sim.ctx, cid)
    return B.records_to_numpy(rec), tabs


def _oracle(circ, coins, noise):
    rec, tab, _ = oracle.run(circ, coins, noise, return_tableau=True)
    return rec, tab


def _assert_tableau_equal(got, want, tag):
    for name, g, w in zip("xzr", got, want):
        assert np.array_equal(g, w), f"{tag}: tableau {name} differs"


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 97, 130])
def test_layered_random_circuits_match_oracle(sim, n):
    for seed in range(4):
        circ = C.random_small_circuit(n, 12 * n + 40, seed=seed + 17 * n)
        coins, noise = S.streams_for(circ, seed, [0])
        rec, tabs = _apply_layered(sim, circ, coins[0], noise[0])
        orec, otab = _oracle(circ, coins[0], noise[0])
        assert np.array_equal(rec[0][:circ.record_words], orec), (n, seed)
        _assert_tableau_equal(tabs[0], otab, f"n={n} seed={seed}")


def test_layered_multi_tableau_batch(sim):
    circ = C.random_small_circuit(40, 600, seed=3)
    shots = 6
    coins, noise = S.streams_for(circ, 9, range(shots))
    rec, tabs = _apply_layered(sim, circ, coins, noise, count=shots)
    for s in range(shots):
        orec, otab = _oracle(circ, coins[s], noise[s])
        assert np.array_equal(rec[s], orec)
        _assert_tableau_equal(tabs[s], otab, f"shot {s}")


@pytest.mark.parametrize("d,p", [(3, 1e-3), (5, 0.02), (7, 1e-3), (9, 0.01), (15, 1e-3)])
def test_layered_surface_code_matches_oracle(sim, d, p):
    circ = C.surface_code_memory(d, p=p)
    coins, noise = S.streams_for(circ, d, [0])
    rec, tabs = _apply_layered(sim, circ, coins[0], noise[0])
    orec, otab = _oracle(circ, coins[0], noise[0])
    assert np.array_equal(rec[0], orec)
    _assert_tableau_equal(tabs[0], otab, f"d={d}")


def test_random_clifford_layers_match_oracle(sim):
    circ = C.random_clifford_layers(200, 30, seed=0)
    coins, noise = S.streams_for(circ, 0, [0])
    rec, tabs = _apply_layered(sim, circ, coins[0], noise[0])
    orec, otab = _oracle(circ, coins[0], noise[0])
    assert np.array_equal(rec[0], orec)
    _assert_tableau_equal(tabs[0], otab, "random clifford")


@pytest.mark.parametrize("engine", [B.ENGINE_RESIDENT, B.ENGINE_LAYERED])
def test_sample_engines_match_oracle(sim, engine):
    circ = C.surface_code_memory(3, p=0.01)
    shots = 300
    coins, noise = S.streams_for(circ, 0, range(shots))
    cid = sim.compile(circ)
    rec = B.records_to_numpy(sim.sample(cid, circ, shots, coins, noise, engine=engine))
    sim.sync()
    orec, _ = oracle.sample(circ, coins, noise, threads=4)
    assert np.array_equal(rec, orec)


@pytest.mark.parametrize("n", [1, 17, 33, 64, 97, 200])
def test_resident_random_circuits_match_oracle(sim, n):
    circ = C.random_small_circuit(n, 10 * n + 30, seed=n)
    shots = 16
    coins, noise = S.streams_for(circ, 1, range(shots))
    cid = sim.compile(circ)
    rec = B.records_to_numpy(sim.sample(cid, circ, shots, coins, noise, engine=B.ENGINE_RESIDENT))
    sim.sync()
    orec, _ = oracle.sample(circ, coins, noise)
    assert np.array_equal(rec, orec)


def test_seeded_streams_match_generator(sim):
    """On-device SplitMix64 streams equal the generator's buffers."""
    circ = C.surface_code_memory(5, p=0.02)
    shots = 64
    coins, noise = S.streams_for(circ, 77, range(10, 10 + shots))
    orec, _ = oracle.sample(circ, coins, noise)
    cid = sim.compile(circ)
    for eng in (B.ENGINE_RESIDENT, B.ENGINE_LAYERED):
        rec = B.records_to_numpy(sim.sample(cid, circ, shots, seed=77, shot_offset=10, engine=eng))
        sim.sync()
        assert np.array_equal(rec, orec), eng


def test_mixed_distance_batch_one_launch(sim):
    """Many circuits of uneven qubit counts in one persistent launch."""
    import torch
    groups, want, bufs = [], [], []
    for d, shots in ((3, 40), (5, 25), (7, 10), (9, 5), (11, 3)):
        T = {"T1": 100e-6, "T2": 80e-6, "t1q": 50e-9, "t2q": 300e-9, "tm": 1e-6}
        circ = C.surface_code_memory(d, t1t2=T)
        cid = sim.compile(circ)
        coins, noise = S.streams_for(circ, 5, range(shots))
        orec, _ = oracle.sample(circ, coins, noise, threads=4)
        rec = sim.record_buffer(shots, circ.record_words)
        dc, dn = sim.to_dev(coins), sim.to_dev(noise)
        bufs += [dc, dn, rec]
        g = B.JobGroup()
        g.circuit_id, g.shots = cid, shots
        g.streams = B.make_streams(B.STREAM_BUFFER, coins=dc, noise=dn)
        g.d_record, g.record_words = rec.data_ptr(), circ.record_words
        groups.append(g)
        want.append((rec, orec))
    B.stab_sample_batch(sim.ctx, groups)
    sim.sync()
    for rec, orec in want:
        assert np.array_equal(B.records_to_numpy(rec), orec)


def test_reset_error_channel_matches_oracle(sim):
    b = C.Builder(6)
    rng = np.random.default_rng(0)
    for _ in range(200):
        k = rng.integers(4)
        q = int(rng.integers(6))
        if k == 0:
            b.gate1(C.H, q)
        elif k == 1:
            b.gate2(C.CX, q, (q + 1) % 6)
        elif k == 2:
            b.reset_error(q, 0.3, 0.2)
        else:
            b.measure(q)
    circ = b.build()
    shots = 32
    coins, noise = S.streams_for(circ, 4, range(shots))
    orec, _ = oracle.sample(circ, coins, noise)
    cid = sim.compile(circ)
    for eng in (B.ENGINE_RESIDENT, B.ENGINE_LAYERED):
        rec = B.records_to_numpy(sim.sample(cid, circ, shots, coins, noise, engine=eng))
        sim.sync()
        assert np.array_equal(rec, orec), eng


def test_empty_and_measure_only(sim):
    b = C.Builder(4)
    b.tick()
    circ = b.build()
    cid = sim.compile(circ)
    rec = sim.sample(cid, circ, 3, np.zeros((3, 1), np.uint64), np.zeros((3, 1), np.uint32))
    sim.sync()
    assert not B.records_to_numpy(rec).any()
    b = C.Builder(70)
    for q in range(70):
        b.measure(q)
    circ = b.build()
    cid = sim.compile(circ)
    for eng in (B.ENGINE_RESIDENT, B.ENGINE_LAYERED):
        rec = sim.sample(cid, circ, 2, np.full((2, 2), 2 ** 64 - 1, np.uint64),
                         np.zeros((2, 1), np.uint32), engine=eng)
        sim.sync()
        assert not B.records_to_numpy(rec).any()


def test_host_validation_errors(sim):
    b = C.Builder(3)
    b.gate2(C.CX, 1, 1)
    with pytest.raises(B.StabError) as e:
        sim.compile(b.build())
    assert e.value.code == B.ERR_ARG
    circ = C.ghz(5)
    cid = sim.compile(circ)
    short = sim.to_dev(np.zeros((2, 1), np.uint64))
    rec = sim.record_buffer(2, 1)
    st = B.make_streams(B.STREAM_BUFFER, coins=short)
    st.coin_words = 0
    with pytest.raises(B.StabError) as e:
        B.stab_sample(sim.ctx, cid, 2, st, rec)
    assert e.value.code == B.ERR_STREAM_SHORT


def _measure_all_after(n, layers, seed):
    """Random Clifford layers without measurement, then one layer measuring
    every qubit: a single measurement layer with many random outcomes."""
    base = C.random_clifford_layers(n, layers, seed=seed, meas_frac=0.0)
    b = C.Builder(n)
    for q in range(n):
        b.measure(q)
    return C.concat([base, b.build()])


def _wave_cases():
    yield "independent", (lambda: (lambda b: ([b.gate1(C.H, q) for q in range(300)],
                                              [b.measure(q) for q in range(300)], b.build())[-1])(C.Builder(300)))()
    yield "shallow", _measure_all_after(300, 2, 1)
    yield "deep", _measure_all_after(160, 12, 2)
    yield "surface", C.surface_code_memory(9, p=5e-3)


def _check_wave_cases(sim):
    for name, circ in _wave_cases():
        coins, noise = S.streams_for(circ, 3, [0])
        rec, tabs = _apply_layered(sim, circ, coins[0], noise[0])
        orec, otab = _oracle(circ, coins[0], noise[0])
        assert np.array_equal(rec[0], orec), name
        _assert_tableau_equal(tabs[0], otab, name)


def test_wave_measurement_layers_match_oracle(sim):
    _check_wave_cases(sim)


def test_wave_list_overflow_fallbacks_match_oracle():
    """Shrunken wave-list capacities force every fallback path of the random
    measurement kernel (pending window, wave size, rowsum-pair list, column
    update list, marking budget)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import tests.test_gpu_parity as t\n"
            "from paper_2507_03092_gb300 import binding as B\n"
            "s = B.Simulator(0)\n"
            "t._check_wave_cases(s)\n"
            "s.close()\nprint('ok')\n")
    for caps in ("8,2,4,4,16", "64,1,2,2,1", "3,1000,1,1,100000", "100,50,100,100,200,3"):
        env = dict(os.environ, STAB_WAVE_CAPS=caps)
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and "ok" in r.stdout, (caps, r.stdout[-2000:], r.stderr[-4000:])


def test_wave_cluster_sizes_match_oracle():
    """The random-measurement kernel spreads each tableau's waves over a
    cluster of CTAs (rank 0 holds the wave state in shared memory); every
    cluster size gives the oracle's records and tableaux, also with shrunken
    list capacities (the fallback loops run cluster-wide too)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import tests.test_gpu_parity as t\n"
            "from paper_2507_03092_gb300 import binding as B\n"
            "s = B.Simulator(0)\n"
            "t._check_wave_cases(s)\n"
            "s.close()\nprint('ok')\n")
    for ncl, caps in (("1", None), ("2", None), ("3", None), ("8", None), ("4", "8,2,4,4,16"),
                      ("8", "64,1,2,2,1")):
        env = dict(os.environ, STAB_RAND_CLUSTER=ncl)
        if caps:
            env["STAB_WAVE_CAPS"] = caps
        r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and "ok" in r.stdout, (ncl, caps, r.stdout[-2000:], r.stderr[-4000:])


_GUARD_CODE = """
import numpy as np
import oracle
from paper_2507_03092_gb300 import binding as B
from paper_2507_03092_gb300 import circuit as C
from paper_2507_03092_gb300 import streams as S
s = B.Simulator(0)
# a layer with random outcomes needs at least two passes of the wave loop (one
# applying a wave, one finding nothing left), so a limit of one pass trips the
# guard: the kernel records a bounds error and returns
g = C.ghz(8)
cid = s.compile(g)
s.sample(cid, g, 4, seed=3, engine=B.ENGINE_LAYERED)
try:
    s.sync()
    print("no error")
except B.StabError as e:
    print("guard", e.code, str(e))
# the context stays usable: a circuit with deterministic outcomes only never
# enters the wave loop and matches the oracle, and the flag was cleared
b = C.Builder(6)
for q in (0, 2, 3):
    b.gate1(C.X, q)
for q in range(6):
    b.measure(q)
det = b.build()
cid2 = s.compile(det)
coins, noise = S.streams_for(det, 1, range(4))
got = B.records_to_numpy(s.sample(cid2, det, 4, coins, noise, engine=B.ENGINE_LAYERED))
s.sync()
want, _ = oracle.sample(det, coins, noise)
print("after", bool(np.array_equal(got, want)))
s.close()
"""


def test_wave_loop_guard_reports_an_error_and_the_context_survives():
    """The wave loop's bound (lowered through STAB_WAVE_CAPS' seventh field)
    fires as a device bounds error that stab_sync reports as
    STAB_ERR_INTERNAL; the kernel returns instead of spinning, and the next
    call on the same context runs normally."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, STAB_WAVE_CAPS="4096,1024,2048,2048,2048,128,1")
    r = subprocess.run([sys.executable, "-c", _GUARD_CODE], cwd=root, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    lines = r.stdout.splitlines()
    guard = [ln for ln in lines if ln.startswith("guard ")]
    assert guard and guard[0].split()[1] == str(B.ERR_INTERNAL) and "bounds" in guard[0], r.stdout
    assert "after True" in lines, r.stdout


@pytest.mark.parametrize("n", [14000, 16400])
def test_layered_wide_measurement_layer(sim, n):
    """One measurement layer of n ops overflows the 4096-entry pending list
    (rebuilt from all items).  n = 16 400 > 16 384: the wave kernel keeps the
    layer's qubit map, item status and stale flags in global memory instead of
    shared memory; n = 14 000 keeps them in shared memory.  Bell pairs joined
    into chains of four make rowsums that touch several rows per random
    measurement."""
    b = C.Builder(n)
    for q in range(n):
        b.gate1(C.H, q)
    for q in range(0, n, 2):
        b.gate2(C.CX, q, q + 1)
    for q in range(1, n - 1, 4):
        b.gate2(C.CX, q, q + 1)
    for q in range(0, n, 3):
        b.gate1(C.S, q)
    for q in range(n):
        b.measure(q)
    circ = b.build()
    coins, noise = S.streams_for(circ, 5, [0])
    rec, tabs = _apply_layered(sim, circ, coins[0], noise[0])
    orec, otab = _oracle(circ, coins[0], noise[0])
    assert np.array_equal(rec[0], orec)
    _assert_tableau_equal(tabs[0], otab, "n=%d" % n)


def test_layered_largest_n_and_one_past_it(sim):
    """The layered engine's largest tableau: n such that one 32-row slice (a
    32-bit x word and z word of every column, 8n bytes) plus 1 KB fits one
    CTA's opt-in shared memory -- 28 928 qubits on GB300.  A sparse circuit
    over the whole range (H and CX on 1200 random qubits and the last one,
    600 of them measured) matches the oracle's records and full tableau; one
    qubit more is refused before anything runs."""
    torch = pytest.importorskip("torch")
    optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin", 232448)
    n = (optin - 1024) // 8
    one_more = C.Builder(n + 1).measure(n).build()
    for bad in (lambda: B.stab_tableau_init(sim.ctx, n + 1, 1),
                lambda: sim.sample(sim.compile(one_more), one_more, 1, seed=1, engine=B.ENGINE_LAYERED)):
        with pytest.raises(B.StabError) as e:
            bad()
        assert e.value.code == B.ERR_UNSUPPORTED
    rng = np.random.default_rng(11)
    qs = [int(q) for q in rng.choice(n - 1, size=1200, replace=False)]
    b = C.Builder(n)
    for q in qs:
        b.gate1(C.H, q)
    for i in range(0, 1200, 2):
        b.gate2(C.CX, qs[i], qs[i + 1])
    for q in qs[:40]:
        b.gate2(C.CX, q, n - 1)
    for q in qs[::3]:
        b.gate1(C.S, q)
    for q in qs[:600] + [n - 1]:
        b.measure(q)
    circ = b.build()
    coins, noise = S.streams_for(circ, 8, [0])
    rec, tabs = _apply_layered(sim, circ, coins[0], noise[0])
    orec, otab = _oracle(circ, coins[0], noise[0])
    assert np.array_equal(rec[0], orec)
    _assert_tableau_equal(tabs[0], otab, f"n={n}")


def _resident_bytes(n):
    """Shared memory of one resident tableau: x and z as [n][2H] words, the
    sign column, per-row counters [64H], the measured-column snapshot [2H],
    pivot-row Paulis [n], per-op flag bytes [n] and 8 words of state."""
    H = (n + 31) // 32
    CW = 2 * H
    return 4 * (2 * n * CW + CW + 64 * H + CW + n + (n + 3) // 4 + 8)


def test_resident_largest_n_and_one_past_it(sim):
    """The resident engine's largest tableau (664 qubits on GB300: its shared
    memory plus 64 bytes fits one CTA's opt-in shared memory) matches the
    oracle over 8 shots of a random circuit with every op kind; one qubit
    more is refused before anything runs."""
    torch = pytest.importorskip("torch")
    optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin", 232448)
    n = max(m for m in range(1, 4096) if _resident_bytes(m) + 64 <= optin)
    one_more = C.random_small_circuit(n + 1, 50, seed=2)
    with pytest.raises(B.StabError) as e:
        sim.sample(sim.compile(one_more), one_more, 4, seed=1, engine=B.ENGINE_RESIDENT)
    assert e.value.code == B.ERR_UNSUPPORTED
    circ = C.random_small_circuit(n, 4 * n, seed=n)
    shots = 8
    coins, noise = S.streams_for(circ, 3, range(shots))
    cid = sim.compile(circ)
    rec = B.records_to_numpy(sim.sample(cid, circ, shots, coins, noise, engine=B.ENGINE_RESIDENT))
    sim.sync()
    orec, _ = oracle.sample(circ, coins, noise, threads=4)
    assert np.array_equal(rec, orec)
