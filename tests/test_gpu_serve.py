"""Served form: requests submitted while others are on the GPU are admitted by
HBM footprint, overlap on the device, and each request's records equal the
records of the same request run alone (and the oracle's)."""
import time

import numpy as np
import pytest

import oracle
from paper_2507_03092_gb300 import binding as B
from paper_2507_03092_gb300 import circuit as C
from paper_2507_03092_gb300 import serve_trace as T
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


def _run_mix(sim, reqs, circs, budget, n_streams=4, spacing=0.0):
    bufs = [sim.record_buffer(sh, circs[d][0].record_words) for d, sh, _ in reqs]
    B.stab_serve_start(sim.ctx, budget, max_inflight=16, n_streams=n_streams, max_batch_requests=8)
    try:
        ids = []
        for (d, sh, seed), buf in zip(reqs, bufs):
            ids.append(B.stab_serve_submit(sim.ctx, circs[d][1], sh, seed, 0, buf))
            if spacing:
                time.sleep(spacing)
        B.stab_serve_drain(sim.ctx, timeout_s=600)
        st = {s["req_id"]: s for s in B.stab_serve_poll(sim.ctx)}
    finally:
        B.stab_serve_stop(sim.ctx)
    assert set(st) == set(ids)
    assert all(s["status"] == 0 for s in st.values())
    for s in st.values():
        assert s["t_submit"] <= s["t_admit"] <= s["t_done"]
    return [B.records_to_numpy(b) for b in bufs]


def test_requests_same_alone_and_in_the_mix(sim):
    dists = (3, 5, 7, 15)
    circs = {d: (c := C.surface_code_memory(d, p=2e-3), sim.compile(c)) for d in dists}
    rng = np.random.default_rng(0)
    reqs = [(int(rng.choice(dists)), int(rng.integers(1, 24)), 500 + i) for i in range(40)]
    mixed = _run_mix(sim, reqs, circs, budget=8 << 30, spacing=0.0005)
    for (d, sh, seed), got in zip(reqs, mixed):
        c, cid = circs[d]
        alone = B.records_to_numpy(sim.sample(cid, c, sh, seed=seed))
        sim.sync()
        assert np.array_equal(got, alone), (d, sh, seed)
    # and every one of them against the oracle, with the generator's streams
    # for the same keys
    for (d, sh, seed), got in zip(reqs, mixed):
        c = circs[d][0]
        coins, noise = S.streams_for(c, seed, range(sh))
        want, _ = oracle.sample(c, coins, noise)
        assert np.array_equal(got, want)


def test_small_budget_still_serves_everything(sim):
    """A budget that admits one request at a time serialises but completes."""
    circs = {3: (c := C.surface_code_memory(3, p=1e-2), sim.compile(c)),
             15: (c2 := C.surface_code_memory(15, p=1e-3), sim.compile(c2))}
    reqs = [(3, 50, 1), (15, 4, 2), (3, 7, 3), (15, 2, 4), (3, 1, 5)]
    one = max(C.surface_code_memory(15).n, 1)
    budget = 60 << 20        # above any single request here, below their sum
    got = _run_mix(sim, reqs, circs, budget=budget, n_streams=2)
    for (d, sh, seed), g in zip(reqs, got):
        c, cid = circs[d]
        alone = B.records_to_numpy(sim.sample(cid, c, sh, seed=seed))
        sim.sync()
        assert np.array_equal(g, alone)
    assert one > 0


def test_oversized_request_rejected_at_submit(sim):
    c = C.surface_code_memory(15)
    cid = sim.compile(c)
    buf = sim.record_buffer(256, c.record_words)
    B.stab_serve_start(sim.ctx, 1 << 20, max_inflight=4, n_streams=2)
    try:
        with pytest.raises(B.StabError) as e:
            B.stab_serve_submit(sim.ctx, cid, 256, 1, 0, buf)
        assert e.value.code == B.ERR_OOM
    finally:
        B.stab_serve_stop(sim.ctx)


def test_short_trace_replay_reports_latency(sim, ):
    import torch
    out = T.replay(sim, B, torch, rate=100.0, duration=0.5, distances=(3, 5, 7, 9), max_shots=16,
                   hbm_budget=4 << 30, n_streams=4)
    assert out["failed"] == 0 and out["requests"] > 10
    assert 0 < out["p50_latency_s"] <= out["p99_latency_s"] < 60
