"""Serving trace: seeded request arrivals and an open-loop replay through the
C-ABI request loop (``stab_serve_*``).

Trace (inputs only): Poisson arrivals at ``rate`` requests/s for ``duration``
seconds (exponential inter-arrival times from a PCG64 stream); each request is
a rotated surface-code Z-memory circuit with distance d uniform over the odd
values 3..31, d rounds, DEPOLARIZE1/2(p) after every H/CNOT, and a shot count
uniform in 1..256.  Its coin and noise streams are the SplitMix64 streams
keyed by (seed = request index + base, shot), generated on the device, so a
request's records do not depend on what else is being served.

Replay: requests are submitted at their arrival times (open loop; a request is
never delayed by the completion of others), the library's scheduler admits
them by HBM footprint into free launch slots and overlaps their work on the
device; latency = completion - arrival.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import circuit as C

DISTANCES = tuple(range(3, 32, 2))


@dataclass
class Request:
    idx: int
    t_arrival: float
    d: int
    shots: int
    seed: int


def make_trace(rate=200.0, duration=60.0, seed=0, distances=DISTANCES, max_shots=256,
               seed_base=1_000_000):
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        d = int(distances[int(rng.integers(len(distances)))])
        shots = int(rng.integers(1, max_shots + 1))
        out.append(Request(len(out), t, d, shots, seed_base + len(out)))
    return out


def compile_circuits(sim, distances=DISTANCES, p=1e-3):
    circs = {}
    for d in distances:
        c = C.surface_code_memory(d, p=p)
        circs[d] = (c, sim.compile(c))
    return circs


def replay(sim, B, torch, rate=200.0, duration=60.0, seed=0, distances=DISTANCES,
           max_shots=256, p=1e-3, hbm_budget=64 << 30, n_streams=16, max_inflight=64,
           max_batch_requests=32, circs=None, keep_records=False):
    """Replay the trace; returns a summary dict (and records if asked)."""
    trace = make_trace(rate, duration, seed, distances, max_shots)
    circs = circs or compile_circuits(sim, distances, p)
    # warm the engines once per distance (allocations, attribute set-up)
    for d in distances:
        c, cid = circs[d]
        rec = sim.record_buffer(1, c.record_words)
        sim.sample(cid, c, 1, seed=1, shot_offset=0, out=rec)
    sim.sync()
    bufs = [sim.record_buffer(r.shots, circs[r.d][0].record_words) for r in trace]
    B.stab_serve_start(sim.ctx, hbm_budget, max_inflight=max_inflight, n_streams=n_streams,
                       max_batch_requests=max_batch_requests)
    ids = {}
    done = {}
    t0 = time.monotonic()
    try:
        for r, buf in zip(trace, bufs):
            now = time.monotonic() - t0
            if r.t_arrival > now:
                time.sleep(r.t_arrival - now)
            rid = B.stab_serve_submit(sim.ctx, circs[r.d][1], r.shots, r.seed, 0, buf)
            ids[rid] = r
            for st in B.stab_serve_poll(sim.ctx):
                done[st["req_id"]] = st
        B.stab_serve_drain(sim.ctx, timeout_s=3600.0)
        for st in B.stab_serve_poll(sim.ctx):
            done[st["req_id"]] = st
    finally:
        B.stab_serve_stop(sim.ctx)
    t_end = time.monotonic() - t0
    lat, qwait, shots = [], [], 0
    bad = 0
    for rid, r in ids.items():
        st = done.get(rid)
        if st is None or st["status"] != 0:
            bad += 1
            continue
        # t_done is CLOCK_MONOTONIC seconds, as is time.monotonic()
        lat.append(st["t_done"] - (t0 + r.t_arrival))
        qwait.append(st["t_admit"] - st["t_submit"])
        shots += r.shots
    lat = np.array(lat)
    last_done = max(st["t_done"] for st in done.values()) - t0 if done else t_end
    out = {
        "workload": f"Poisson {rate:g} req/s over {duration:g} s, d uniform odd {distances[0]}..{distances[-1]}, "
                    f"d rounds, depolarizing p={p:g}, shots uniform 1..{max_shots}",
        "requests": len(trace), "failed": bad, "shots": shots,
        "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_admission_wait_s": float(np.mean(qwait)) if qwait else None,
        "makespan_s": float(last_done),
        "throughput_shots_per_s": shots / last_done if last_done > 0 else None,
        "offered_shots_per_s": sum(r.shots for r in trace) / duration,
        "config": {"hbm_budget_bytes": int(hbm_budget), "n_streams": n_streams,
                   "max_inflight": max_inflight, "max_batch_requests": max_batch_requests},
    }
    if keep_records:
        out["records"] = {r.idx: B.records_to_numpy(buf) for r, buf in zip(trace, bufs)}
        out["trace"] = trace
    return out


def saturated(sim, B, torch, n_requests=2000, seed=0, distances=DISTANCES, max_shots=256, p=1e-3,
              hbm_budget=64 << 30, n_streams=16, max_inflight=64, max_batch_requests=32, circs=None):
    """Capacity: the first ``n_requests`` requests of the trace submitted all
    at once (an offered rate far above what the loop can serve), shots/s =
    their shots / the time until the last one completes."""
    trace = make_trace(200.0, 2.0 * n_requests / 200.0 + 10.0, seed, distances, max_shots)[:n_requests]
    circs = circs or compile_circuits(sim, distances, p)
    bufs = [sim.record_buffer(r.shots, circs[r.d][0].record_words) for r in trace]
    B.stab_serve_start(sim.ctx, hbm_budget, max_inflight=max_inflight, n_streams=n_streams,
                       max_batch_requests=max_batch_requests)
    done = {}
    t0 = time.monotonic()
    try:
        for r, buf in zip(trace, bufs):
            B.stab_serve_submit(sim.ctx, circs[r.d][1], r.shots, r.seed, 0, buf)
        B.stab_serve_drain(sim.ctx, timeout_s=3600.0)
        for st in B.stab_serve_poll(sim.ctx):
            done[st["req_id"]] = st
    finally:
        B.stab_serve_stop(sim.ctx)
    ok = [st for st in done.values() if st["status"] == 0]
    span = max(st["t_done"] for st in ok) - t0 if ok else float("nan")
    shots = sum(r.shots for r in trace)
    lat = np.array([st["t_done"] - st["t_submit"] for st in ok])
    return {"requests": len(trace), "failed": len(trace) - len(ok), "shots": shots,
            "makespan_s": span, "capacity_shots_per_s": shots / span if span > 0 else None,
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "offered": "all requests submitted at t = 0"}


def plain(sim, B, torch, n_requests=200, seed=0, distances=DISTANCES, max_shots=256, p=1e-3, circs=None):
    """The plain path on the same mix: one tableau per launch sequence (the
    layered engine, one shot per stab_sample call, synchronised), timed on
    one shot of each of the first ``n_requests`` requests; a request's time is
    its shot count times that per-shot time, so shots/s = shots / sum of
    request times over the sample."""
    trace = make_trace(200.0, 2.0 * n_requests / 200.0 + 10.0, seed, distances, max_shots)[:n_requests]
    circs = circs or compile_circuits(sim, distances, p)
    per_d = {}
    for d in sorted({r.d for r in trace}):
        c, cid = circs[d]
        rec = sim.record_buffer(1, c.record_words)
        sim.sample(cid, c, 1, seed=1, engine=B.ENGINE_LAYERED, out=rec)     # warm-up
        sim.sync()
        t0 = time.perf_counter()
        for k in range(3):
            sim.sample(cid, c, 1, seed=2, shot_offset=k, engine=B.ENGINE_LAYERED, out=rec)
            sim.sync()
        per_d[d] = (time.perf_counter() - t0) / 3
    tot_t = sum(r.shots * per_d[r.d] for r in trace)
    shots = sum(r.shots for r in trace)
    return {"requests_sampled": len(trace), "shots": shots, "plain_shots_per_s": shots / tot_t,
            "per_shot_ms": {str(d): round(1e3 * v, 3) for d, v in per_d.items()},
            "method": "layered engine, one shot per synchronised stab_sample call, host wall time"}
