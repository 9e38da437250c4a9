"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times: bit-exact records (and tableaux where the oracle can follow)
against the CPU oracle, or properties that hold at any size."""
import os

import numpy as np
import pytest

import oracle
from paper_2507_03092_gb300 import binding as B
from paper_2507_03092_gb300 import circuit as C
from paper_2507_03092_gb300 import streams as S

pytestmark = pytest.mark.gpu
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def sim():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = B.Simulator(0)
    yield s
    s.close()


def test_config1_d3_1024_shots_both_engines(sim):
    circ = C.surface_code_memory(3, p=1e-3)
    coins, noise = S.streams_for(circ, 0, range(1024))
    want, _ = oracle.sample(circ, coins, noise, threads=THREADS)
    cid = sim.compile(circ)
    for eng in (B.ENGINE_RESIDENT, B.ENGINE_LAYERED):
        got = B.records_to_numpy(sim.sample(cid, circ, 1024, coins, noise, engine=eng))
        sim.sync()
        assert np.array_equal(got, want), eng


def test_config2_random_clifford_n1000_200_layers(sim):
    circ = C.random_clifford_layers(1000, 200, seed=0)
    coins, noise = S.streams_for(circ, 0, [0])
    want, wtab, st = oracle.run(circ, coins[0], noise[0], return_tableau=True)
    cid = sim.compile(circ)
    B.stab_tableau_init(sim.ctx, circ.n, 1)
    rec = sim.record_buffer(1, circ.record_words)
    B.stab_apply_circuit(sim.ctx, cid, B.make_streams(B.STREAM_BUFFER, coins=sim.to_dev(coins),
                                                      noise=sim.to_dev(noise)), rec)
    sim.sync()
    assert np.array_equal(B.records_to_numpy(rec)[0], want)
    for g, w in zip(B.stab_get_tableau(sim.ctx, 0, circ.n), wtab):
        assert np.array_equal(g, w)
    assert st["n_meas_random"] > 10000          # the workload is dominated by random outcomes


def _golden(name):
    import json
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", name)) as fh:
        return json.load(fh)


def _digest(words):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(words, "<u8").tobytes()).hexdigest()


def test_config3_d71_noiseless_full_record_matches_golden(sim):
    """All 362 881 outcomes of the noiseless d=71 circuit, shot 0 of seeds 0
    and 1 (device-generated seeded streams), against the oracle's records
    stored as digests by tests/golden/make_golden.py (oracle only)."""
    circ = C.surface_code_memory(71)
    cid = sim.compile(circ)
    for seed in (0, 1):
        gold = _golden(f"d71_noiseless_seed{seed}.json")
        rec = B.records_to_numpy(sim.sample(cid, circ, 1, seed=seed, engine=B.ENGINE_LAYERED))
        sim.sync()
        assert rec.shape[1] == gold["record_words"]
        bits = oracle.record_bits(rec, circ.n_meas)[0]
        assert int(bits.sum()) == gold["ones"], seed
        assert gold["detectors_fired"] == 0
        assert _digest(rec[0]) == gold["record_sha256"], seed


def _check_serve_golden(recs, gold):
    for got, req in zip(recs, gold["requests"]):
        assert got.shape == (req["shots"], req["record_words"]), req["d"]
        bad = [s for s in range(req["shots"]) if _digest(got[s])[:32] != req["shot_sha256"][s]]
        assert not bad, (req["d"], bad[:10])


def test_config5_largest_requests_match_oracle_alone_and_served(sim):
    """The largest requests of the serving workload -- d=31 with 256 shots and
    d=29 with 200 shots, DEPOLARIZE p=1e-3, seeded streams keyed by (request
    seed, shot) -- through stab_sample and through the serving loop (mixed
    with smaller requests), every shot's record against the oracle's (digests
    written by tests/golden/make_golden.py)."""
    gold = _golden("serve_largest.json")
    circs = {}
    for req in gold["requests"]:
        c = C.surface_code_memory(req["d"], p=1e-3)
        circs[req["d"]] = (c, sim.compile(c))
    alone = []
    for req in gold["requests"]:
        c, cid = circs[req["d"]]
        alone.append(B.records_to_numpy(sim.sample(cid, c, req["shots"], seed=req["seed"])))
        sim.sync()
    _check_serve_golden(alone, gold)
    # served: the two largest requests among smaller ones of other distances
    small = {d: (c := C.surface_code_memory(d, p=1e-3), sim.compile(c)) for d in (3, 9, 17)}
    bufs, ids, order = [], [], []
    B.stab_serve_start(sim.ctx, 16 << 30, max_inflight=16, n_streams=4, max_batch_requests=8)
    try:
        for k, (d, sh) in enumerate([(3, 40), (9, 17), (17, 5), (3, 100)]):
            c, cid = small[d]
            buf = sim.record_buffer(sh, c.record_words)
            ids.append(B.stab_serve_submit(sim.ctx, cid, sh, 70 + k, 0, buf))
            bufs.append(buf)
            order.append(None)
            if k == 1:
                for j, req in enumerate(gold["requests"]):
                    c, cid = circs[req["d"]]
                    buf = sim.record_buffer(req["shots"], c.record_words)
                    ids.append(B.stab_serve_submit(sim.ctx, cid, req["shots"], req["seed"], 0, buf))
                    bufs.append(buf)
                    order.append(j)
        B.stab_serve_drain(sim.ctx, timeout_s=600)
        st = {x["req_id"]: x for x in B.stab_serve_poll(sim.ctx)}
    finally:
        B.stab_serve_stop(sim.ctx)
    assert set(st) == set(ids) and all(x["status"] == 0 for x in st.values())
    served = [None] * len(gold["requests"])
    for buf, j in zip(bufs, order):
        if j is not None:
            served[j] = B.records_to_numpy(buf)
    _check_serve_golden(served, gold)


def test_config3_d71_noiseless_detectors_all_zero(sim):
    circ = C.surface_code_memory(71)
    cid = sim.compile(circ)
    for seed in (0, 1):
        rec = B.records_to_numpy(sim.sample(cid, circ, 1, seed=seed, engine=B.ENGINE_LAYERED))
        sim.sync()
        bits = oracle.record_bits(rec, circ.n_meas)[0]
        det = np.array([np.bitwise_xor.reduce(bits[d]) for d in circ.meta["detectors"]])
        assert not det.any()
        assert int(np.bitwise_xor.reduce(bits[circ.meta["observable"]])) == 0
        # round-1 X-ancilla outcomes follow the coins (random), so records differ by seed
        assert bits.any()


def test_config3_d71_noisy_prefix_bit_exact(sim):
    """The d=71 noisy circuit's first rounds on the layered engine the
    benchmark times, against the oracle: records and the full tableau."""
    full = C.surface_code_memory(71, p=1e-3)
    pre = C.prefix(full, full.meta["round_end"][1])        # reset + 2 syndrome rounds
    coins, noise = S.streams_for(full, 0, [0])
    want, wtab, _ = oracle.run(pre, coins[0], noise[0], return_tableau=True)
    cid = sim.compile(pre)
    B.stab_tableau_init(sim.ctx, pre.n, 1)
    rec = sim.record_buffer(1, pre.record_words)
    B.stab_apply_circuit(sim.ctx, cid, B.make_streams(B.STREAM_BUFFER, coins=sim.to_dev(coins),
                                                      noise=sim.to_dev(noise)), rec)
    sim.sync()
    assert np.array_equal(B.records_to_numpy(rec)[0], want)
    for g, w in zip(B.stab_get_tableau(sim.ctx, 0, pre.n), wtab):
        assert np.array_equal(g, w)
    # and the full noisy circuit: detector flips are sparse (p = 1e-3)
    cidf = sim.compile(full)
    recf = B.records_to_numpy(sim.sample(cidf, full, 1, coins, noise, engine=B.ENGINE_LAYERED))
    sim.sync()
    bits = oracle.record_bits(recf, full.n_meas)[0]
    det = np.array([np.bitwise_xor.reduce(bits[d]) for d in full.meta["detectors"]])
    assert 0 < det.mean() < 0.05


def test_config4_4096_mixed_distance_shots_one_batch_call(sim):
    """4096 shots of five distances in one stab_sample_batch call (small
    tableaux in one persistent resident launch, d = 11 on the layered engine)."""
    T = {"T1": 100e-6, "T2": 80e-6, "t1q": 50e-9, "t2q": 300e-9, "tm": 1e-6}
    dists = S.shot_distances(0, 4096)
    groups, checks, keep = [], [], []
    for d in (3, 5, 7, 9, 11):
        shots = np.flatnonzero(dists == d)
        circ = C.surface_code_memory(d, t1t2=T)
        coins, noise = S.streams_for(circ, 100 + d, shots)
        want, _ = oracle.sample(circ, coins, noise, threads=THREADS)
        cid = sim.compile(circ)
        rec = sim.record_buffer(len(shots), circ.record_words)
        dc, dn = sim.to_dev(coins), sim.to_dev(noise)
        keep += [dc, dn]
        g = B.JobGroup()
        g.circuit_id, g.shots = cid, len(shots)
        g.streams = B.make_streams(B.STREAM_BUFFER, coins=dc, noise=dn)
        g.d_record, g.record_words = rec.data_ptr(), circ.record_words
        groups.append(g)
        checks.append((rec, want))
    B.stab_sample_batch(sim.ctx, groups)
    sim.sync()
    for rec, want in checks:
        assert np.array_equal(B.records_to_numpy(rec), want)


def test_random_wide_benchmark_matches_oracle(sim):
    circ = C.random_wide_benchmark(96, 96, seed=1)
    coins, noise = S.streams_for(circ, 2, [0])
    want, wtab, _ = oracle.run(circ, coins[0], noise[0], return_tableau=True)
    cid = sim.compile(circ)
    B.stab_tableau_init(sim.ctx, circ.n, 1)
    rec = sim.record_buffer(1, circ.record_words)
    B.stab_apply_circuit(sim.ctx, cid, B.make_streams(B.STREAM_BUFFER, coins=sim.to_dev(coins),
                                                      noise=sim.to_dev(noise)), rec)
    sim.sync()
    assert np.array_equal(B.records_to_numpy(rec)[0], want)
    for g, w in zip(B.stab_get_tableau(sim.ctx, 0, circ.n), wtab):
        assert np.array_equal(g, w)


def test_config3_d71_noisy_full_record_matches_golden(sim):
    """All 362 881 outcomes of the full d=71 noisy circuit (shot 0, seed 0)
    against the oracle's record, stored as a digest by
    tests/golden/make_golden.py (oracle only)."""
    import hashlib
    import json
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", "d71_noisy_seed0.json")) as fh:
        gold = json.load(fh)
    circ = C.surface_code_memory(71, p=1e-3)
    coins, noise = S.streams_for(circ, 0, [0])
    cid = sim.compile(circ)
    rec = B.records_to_numpy(sim.sample(cid, circ, 1, coins, noise, engine=B.ENGINE_LAYERED))
    sim.sync()
    assert rec.shape[1] == gold["record_words"]
    bits = oracle.record_bits(rec, circ.n_meas)[0]
    assert int(bits.sum()) == gold["ones"]
    det = [int(np.bitwise_xor.reduce(bits[d])) for d in circ.meta["detectors"]]
    assert sum(det) == gold["detectors_fired"]
    assert hashlib.sha256(np.ascontiguousarray(rec[0], "<u8").tobytes()).hexdigest() == gold["record_sha256"]
