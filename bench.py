#!/usr/bin/env python3
"""Benchmark: rotated surface-code Z-memory at distance 71 (10081 qubits,
71 syndrome rounds, DEPOLARIZE1/2 p=1e-3 after every H/CNOT), one shot per
step, simulated end to end through the C ABI (stab_sample, layered engine):
tableau init, every Clifford layer, noise, measurement and reset.

Prints ONE JSON line: gate+measure ops/s (value: inputs resident in HBM;
e2e: host buffers through stab_sample_host), the dominant kernel's roofline,
the CPU oracle on a bounded sample, clocks, kernel launches, the batched
(mixed-distance, one persistent launch) vs plain shots/s comparison and, at
N = 1, the 60 s serving trace (p50/p99 latency, shots/s).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--serve | --no-serve]

Under torchrun (N > 1) every rank simulates its own shots on its own GPU
(replicas; no collective on the data path); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_03092_gb300 import circuit as C  # noqa: E402
from paper_2507_03092_gb300 import streams as S  # noqa: E402

METRIC = "surface-code d=71 gate+measure ops/s"

# DRAM bytes (read + write) per launch from one ncu capture of the d=71 step,
# valid only while the CUDA source the capture was taken of is unchanged: each
# entry records the SHA-256 (first 16 hex digits) of the source files, and a
# kernel whose sources changed since reports traffic null.
NCU_TRAFFIC = {
    "k_meas_rand": {"bytes_per_launch": 11.948e6, "src_sha": "5d8a546e25319846",
                    "tag": "ncu capture without cache flushing, mean over the 2 launches of a d=71 step "
                           "(9.51 MB read + 14.39 MB written; the other 70 measurement layers have no "
                           "random op and launch no wave kernel)"},
    "k_gate_run": {"bytes_per_launch": 64.20e6, "src_sha": "5d8a546e25319846",
                   "tag": "ncu capture without cache flushing, steady syndrome-round launch "
                          "(6.80 MB read + 57.40 MB written, the writes mostly dirty lines evicted from L2)"},
}
KERNEL_SOURCES = ("paper_2507_03092_gb300/csrc/layered.cu", "paper_2507_03092_gb300/csrc/device_common.cuh",
                  "paper_2507_03092_gb300/csrc/internal.h")


def kernel_source_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """(bytes per launch, tag) of the committed capture, or (None, reason)."""
    tr = NCU_TRAFFIC.get(kernel)
    if not tr:
        return None, "no capture"
    if tr["src_sha"] != kernel_source_sha():
        return None, "kernel changed since its ncu capture"
    return tr["bytes_per_launch"], tr["tag"]


L2_FLUSH_BYTES = 512 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def l2_sweep(sim, B, torch):
    """Measured L2 read + write bandwidth: the library's copy probe over
    working sets of 8..64 MB (two buffers of half the size each, well below
    the L2 size), many passes in one launch; the best size is the L2 peak.
    One size far above L2 (2 GiB) gives the same probe's HBM figure for
    comparison with the measured copy peak."""
    props = torch.cuda.get_device_properties(sim.device)
    l2_bytes = int(getattr(props, "L2_cache_size", 0) or 0)
    per = {}
    for mb in (8, 16, 32, 48, 64, 80, 96, 112, 128):
        per[mb] = B.stab_probe_copy(sim.ctx, mb << 20, 200 if mb <= 64 else 50)
    best_mb = max(per, key=per.get)
    # largest working set that still gets at least 90 % of the best figure
    knee = max(mb for mb, v in per.items() if v >= 0.9 * per[best_mb])
    hbm_probe = B.stab_probe_copy(sim.ctx, 2 << 30, 5)
    return {"l2_gbs": per[best_mb], "best_working_set_mb": best_mb, "l2_effective_bytes": knee << 20,
            "per_working_set_gbs": {str(k): round(v, 1) for k, v in per.items()},
            "l2_cache_bytes": l2_bytes, "hbm_gbs_same_probe": hbm_probe,
            "method": "stab_probe_copy: 16-byte ld/st.cg copy, 200 passes (50 above 64 MB) in one "
                      "launch over two buffers of half the working set, CUDA events; read + write bytes; "
                      "l2_effective_bytes = the largest working set still within 10 % of the best"}


def roof_bound(working_set_bytes, l2_bytes):
    """'l2' when one launch's working set fits the L2 cache (the largest
    working set the copy probe still runs at L2 speed), else 'hbm'."""
    return "l2" if l2_bytes and working_set_bytes <= l2_bytes else "hbm"


def tableau_bytes(n):
    """(column-packed copy, row-packed copy) bytes of one n-qubit tableau."""
    H = (n + 31) // 32
    Hr = (H + 3) // 4 * 4
    return 8 * 2 * H * n, 4 * 64 * H * 2 * Hr


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle
def oracle_ops_per_s(circ, coins, noise, budget_s=15.0):
    """Time the CPU oracle on a prefix of the circuit made of whole syndrome
    rounds, sized to about ``budget_s`` seconds from a one-round probe.
    Returns (gate+measure ops/s, description, seconds)."""
    import oracle
    ends = circ.meta.get("round_end") or [len(circ.ops)]
    pre = C.prefix(circ, ends[0])
    t0 = time.perf_counter()
    oracle.run(pre, coins, noise)
    t_one = time.perf_counter() - t0
    k = int(max(1, min(len(ends), budget_s // max(t_one, 1e-6))))
    if k > 1:
        pre = C.prefix(circ, ends[k - 1])
        t0 = time.perf_counter()
        oracle.run(pre, coins, noise)
        dt = time.perf_counter() - t0
    else:
        dt = t_one
    ops = C.gate_measure_ops(pre)
    desc = (f"first {k} of {len(ends)} syndrome rounds of the d={circ.meta.get('d')} circuit "
            f"({ops} gate+measure ops, {len(pre.ops)} ops incl. noise), 1 thread, {dt:.2f} s")
    return ops / dt, desc, dt


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    d = args.d
    circ = C.surface_code_memory(d, p=args.p)
    coins, noise = S.streams_for(circ, 0, [0])
    for _ in range(args.warmup):
        oracle_ops_per_s(circ, coins[0], noise[0], budget_s=args.ref_step_s)
    vals, descs, secs = [], [], []
    for _ in range(args.steps):
        v, dsc, dt = oracle_ops_per_s(circ, coins[0], noise[0], budget_s=args.ref_step_s)
        vals.append(v)
        descs.append(dsc)
        secs.append(dt)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ops/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"rotated surface-code Z-memory d={d}, {d} rounds, "
                               f"depolarizing p={args.p}, single shot", "d": d, "n": circ.n},
        "cpu_baseline": {"value": value, "unit": "ops/s", "cores": 1, "kind": "oracle",
                         "sample": descs[-1]},
        "e2e": {"value": value, "unit": "ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batched vs plain
C4_T1T2 = {"T1": 100e-6, "T2": 80e-6, "t1q": 50e-9, "t2q": 300e-9, "tm": 1e-6}
C4_DISTANCES = (3, 5, 7, 9, 11)


def batched_vs_plain(sim, B, torch, shots=4096, plain_shots=64, seed=0, autotune=True, reps=3):
    T = C4_T1T2
    dists = S.shot_distances(seed, shots)
    groups, keep, circs = [], [], {}
    for d in C4_DISTANCES:
        cnt = int(np.count_nonzero(dists == d))
        circ = C.surface_code_memory(d, t1t2=T)
        cid = sim.compile(circ)
        circs[d] = (circ, cid)
        rec = sim.record_buffer(cnt, circ.record_words)
        g = B.JobGroup()
        g.circuit_id, g.shots = cid, cnt
        g.streams = B.make_streams(B.STREAM_SEEDED, seed=seed + d, shot_offset=0)
        g.d_record, g.record_words = rec.data_ptr(), circ.record_words
        groups.append(g)
        keep.append(rec)
    if autotune:
        B.stab_autotune(sim.ctx, [circs[d][1] for d in circs], 256)
    tunes = {d: B.stab_get_tune(sim.ctx, circs[d][0].n) for d in circs}
    for _ in range(2):        # warm-up (as in gpu_rates)
        B.stab_sample_batch(sim.ctx, groups)
        sim.sync()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.stab_sample_batch(sim.ctx, groups)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    sim.sync()
    batched = shots / float(np.median(ts))
    # plain: one tableau per launch sequence (layered engine, one shot per call),
    # on a proportional subset of the same mix
    per_d = {d: max(1, int(round(plain_shots * np.count_nonzero(dists == d) / shots))) for d in circs}
    tot = 0.0
    n_plain = 0
    for d, k in per_d.items():
        circ, cid = circs[d]
        rec = sim.record_buffer(1, circ.record_words)
        for _ in range(2):    # warm-up (as in gpu_rates)
            sim.sample(cid, circ, 1, seed=seed + d, engine=B.ENGINE_LAYERED, out=rec)
            sim.sync()
        t0 = time.perf_counter()
        for s in range(k):
            sim.sample(cid, circ, 1, seed=seed + d, shot_offset=s, engine=B.ENGINE_LAYERED, out=rec)
        sim.sync()
        tot += (time.perf_counter() - t0) * (np.count_nonzero(dists == d) / k)
        n_plain += k
    plain = shots / tot
    return {"workload": "4096 shots, d uniform in {3,5,7,9,11}, d rounds, twirled T1/T2 Pauli noise; "
                        "one stab_sample_batch call (d <= 9: one persistent resident launch, autotuned; "
                        "d = 11: layered engine)",
            "batched_shots_per_s": batched, "plain_shots_per_s": plain,
            "speedup": batched / plain, "plain_sample_shots": n_plain,
            "tune": {str(k): v for k, v in tunes.items()}}


def oracle_batched(shots=4096, per_d=64, seed=0, cores=None):
    """The batched workload on the CPU oracle: the same circuits and streams
    (shot s of distance d keyed by (seed + d, s), as the device's seeded mode),
    a bounded sample of ``per_d`` shots per distance, timed on 1 host thread and
    on ``cores`` threads (all host cores by default); shots/s over the whole
    mix, each distance's time scaled by its share of the shots."""
    import oracle
    cores = cores or os.cpu_count() or 1
    dists = S.shot_distances(seed, shots)
    t1 = tn = 0.0
    n_sample = 0
    for d in C4_DISTANCES:
        cnt = int(np.count_nonzero(dists == d))
        if cnt == 0:
            continue
        k = min(per_d, cnt)
        circ = C.surface_code_memory(d, t1t2=C4_T1T2)
        coins, noise = S.streams_for(circ, seed + d, range(k))
        t0 = time.perf_counter()
        r1, _ = oracle.sample(circ, coins, noise, threads=1)
        t1 += (time.perf_counter() - t0) * cnt / k
        t0 = time.perf_counter()
        rn, _ = oracle.sample(circ, coins, noise, threads=cores)
        tn += (time.perf_counter() - t0) * cnt / k
        if not np.array_equal(r1, rn):
            raise RuntimeError("oracle records differ between thread counts")
        n_sample += k
    return {"kind": "oracle", "one_core_shots_per_s": shots / t1, "all_cores_shots_per_s": shots / tn,
            "cores": cores,
            "sample": f"{n_sample} shots ({per_d} per distance) of the {shots}-shot mix, "
                      f"each distance's time scaled by its share of the shots"}


# ------------------------------------------------------------------ per-config rates
def tick_prefixes(circ):
    """Op counts at the TICKs of a circuit (whole layers / rounds as prefixes)."""
    return [int(i) + 1 for i in np.flatnonzero(circ.ops["kind"] == C.TICK)] or [len(circ.ops)]


def oracle_prefix_rate(circ, coins, noise, budget_s, prefixes=None):
    """The oracle, one thread, on the longest whole-round prefix of ``circ``
    that fits about ``budget_s`` seconds (sized from a one-round probe).
    Returns (gate+measure ops/s, measurements/s, description)."""
    import oracle
    ends = prefixes or tick_prefixes(circ)
    pre = C.prefix(circ, ends[0])
    t0 = time.perf_counter()
    oracle.run(pre, coins, noise)
    t_one = time.perf_counter() - t0
    k = int(max(1, min(len(ends), budget_s // max(t_one, 1e-6))))
    pre = C.prefix(circ, ends[k - 1])
    t0 = time.perf_counter()
    oracle.run(pre, coins, noise)
    dt = time.perf_counter() - t0
    kinds = pre.ops["kind"]
    n_meas = int(np.count_nonzero(np.isin(kinds, (C.M, C.R, C.MPP))))
    ops = C.gate_measure_ops(pre)
    return ops / dt, n_meas / dt, (f"first {k} of {len(ends)} rounds ({ops} gate+measure ops), "
                                   f"1 thread, {dt:.2f} s")


def gpu_rates(sim, B, torch, circ, shots, flush, reps=3, engine=None, seed=0):
    """Device-timed shots of ``circ`` through stab_sample (device-resident
    streams, L2 flushed between reps): shots/s, gates/s, measurements/s,
    gate+measure ops/s, and the ms per call."""
    eng = B.ENGINE_AUTO if engine is None else engine
    cid = sim.compile(circ)
    coins, noise = S.streams_for(circ, seed, range(shots))
    dc, dn = sim.to_dev(coins), sim.to_dev(noise)
    rec = sim.record_buffer(shots, circ.record_words)
    st = B.make_streams(B.STREAM_BUFFER, coins=dc, noise=dn)
    for _ in range(2):        # warm-up: allocation, the circuit's deterministic layers, graph capture
        B.stab_sample(sim.ctx, cid, shots, st, rec, eng)
        sim.sync()
    ts = []
    for i in range(reps):
        flush.fill_(i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.stab_sample(sim.ctx, cid, shots, st, rec, eng)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    sim.sync()
    t = float(np.median(ts))
    kinds = circ.ops["kind"]
    n_g = int(np.count_nonzero(np.isin(kinds, C.ONE_QUBIT_GATES + C.TWO_QUBIT_GATES)))
    n_m = int(np.count_nonzero(np.isin(kinds, (C.M, C.R, C.MPP))))
    sim.release(cid)
    return {"shots_per_s": shots / t, "gates_per_s": n_g * shots / t, "measurements_per_s": n_m * shots / t,
            "ops_per_s": (n_g + n_m) * shots / t, "ms_per_call": 1e3 * t, "shots": shots}, (coins, noise)


def config_suite(sim, B, torch, flush, cpu=True):
    """The other workloads at their stated sizes, with the oracle beside each:
    C1 (d=3, 1024 shots; oracle on 1 thread and all host threads), C2
    (n=1000, 200 random Clifford layers, one tableau), C3 noiseless (d=71,
    one shot) and the random n-wide, n-round H/S/CX/M/R benchmark (Sec. 4.1)
    at three widths."""
    import oracle
    cores = os.cpu_count() or 1
    out = {}
    stage("configs: C1")
    c1 = C.surface_code_memory(3, p=1e-3)
    g, (coins, noise) = gpu_rates(sim, B, torch, c1, 1024, flush)
    if cpu:
        t0 = time.perf_counter()
        oracle.sample(c1, coins, noise, threads=1)
        t1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.sample(c1, coins, noise, threads=cores)
        tn = time.perf_counter() - t0
        g["cpu_baseline"] = {"kind": "oracle", "one_core_shots_per_s": 1024 / t1,
                             "all_cores_shots_per_s": 1024 / tn, "cores": cores, "sample": "all 1024 shots"}
    out["c1_d3_1024_shots"] = g
    stage("configs: C2")
    c2 = C.random_clifford_layers(1000, 200, seed=0)
    g, (coins, noise) = gpu_rates(sim, B, torch, c2, 1, flush, engine=B.ENGINE_LAYERED)
    if cpu:
        ops, meas, desc = oracle_prefix_rate(c2, coins[0], noise[0], 10.0)
        g["cpu_baseline"] = {"kind": "oracle", "ops_per_s": ops, "measurements_per_s": meas, "cores": 1,
                             "sample": desc}
    out["c2_random_clifford_n1000_200_layers"] = g
    stage("configs: C3 noiseless")
    c3 = C.surface_code_memory(71)
    g, (coins, noise) = gpu_rates(sim, B, torch, c3, 1, flush, engine=B.ENGINE_LAYERED)
    if cpu:
        ops, meas, desc = oracle_prefix_rate(c3, coins[0], noise[0], 8.0, c3.meta["round_end"])
        g["cpu_baseline"] = {"kind": "oracle", "ops_per_s": ops, "measurements_per_s": meas, "cores": 1,
                             "sample": desc}
    out["c3_d71_noiseless"] = g
    wide = {}
    for n in (256, 1024, 2048):
        stage(f"configs: random n-wide n={n}")
        cw = C.random_wide_benchmark(n, n, seed=1)
        g, (coins, noise) = gpu_rates(sim, B, torch, cw, 1, flush, reps=2, engine=B.ENGINE_LAYERED)
        if cpu:
            ops, meas, desc = oracle_prefix_rate(cw, coins[0], noise[0], 4.0)
            g["cpu_baseline"] = {"kind": "oracle", "ops_per_s": ops, "measurements_per_s": meas, "cores": 1,
                                 "sample": desc}
        wide[str(n)] = g
    out["random_wide_n_rounds"] = wide
    return out


# ------------------------------------------------------------------ ranks
def shot_indices(rank: int, steps: int, warmup: int) -> list:
    """Stream shot indices of one rank: every rank simulates its own shots
    (replicas), so the ranges are disjoint."""
    return [rank * (steps + warmup) + s for s in range(steps + warmup)]


def aggregate(t_local_s: float, ops_per_step: int, steps: int, world: int, dist=None, device=None):
    """Whole-job throughput: all ranks' ops over the slowest rank's time."""
    t = t_local_s
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t_local_s], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return ops_per_step * steps * world / t, t


# ------------------------------------------------------------------ main arm
def stage(msg):
    """Progress marker on stderr (the JSON line is the only stdout output)."""
    print(f"[bench] {time.strftime('%H:%M:%S')} {msg}", file=sys.stderr, flush=True)


def main():
    faulthandler.enable()            # a fatal signal prints the Python stack to stderr
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--d", type=int, default=71)
    ap.add_argument("--p", type=float, default=1e-3)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="replay the serving trace (p50/p99) also when N > 1 (it runs by default at N = 1)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving trace")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' rates")
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--only", choices=["batched"], default=None,
                    help="run one workload alone (for profiling): 'batched' = the 4096-shot mixed-distance "
                         "batch, default launch shapes, one warm-up and one timed call")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2507_03092_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.only == "batched":
        sim = B.Simulator(local)
        res = batched_vs_plain(sim, B, torch, plain_shots=5, autotune=False, reps=1)
        sim.close()
        print(json.dumps({"only": "batched", "batched": res}), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    d, p = args.d, args.p
    circ = C.surface_code_memory(d, p=p)
    ops_per_step = C.gate_measure_ops(circ)
    kinds_ = circ.ops["kind"]
    n_gates = int(np.count_nonzero(np.isin(kinds_, C.ONE_QUBIT_GATES + C.TWO_QUBIT_GATES)))
    n_meas_ops = int(np.count_nonzero(np.isin(kinds_, (C.M, C.R, C.MPP))))
    n_m_ops = int(np.count_nonzero(np.isin(kinds_, (C.M, C.MPP))))
    n_r_ops = int(np.count_nonzero(kinds_ == C.R))
    K, W = args.steps, args.warmup
    shots_idx = shot_indices(rank, K, W)
    coins, noise = S.streams_for(circ, 0, shots_idx)

    sim = B.Simulator(local)
    cid = sim.compile(circ)
    info = sim.info(cid)
    dc, dn = sim.to_dev(coins), sim.to_dev(noise)
    rec = sim.record_buffer(K + W, circ.record_words)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=sim.device)

    def step(s, profile=False):
        st = B.make_streams(B.STREAM_BUFFER, coins=dc[s:s + 1], noise=dn[s:s + 1])
        B.stab_sample(sim.ctx, cid, 1, st, rec[s:s + 1], B.ENGINE_LAYERED)

    for s in range(W):
        flush.fill_(s)
        step(s)
        # (untimed: each warm-up step ends before the next starts, so the
        # engine has learned the circuit's deterministic measurement layers
        # from the first one and captured its launch graph before timing)
        sim.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    B.stab_launch_count(sim.ctx, reset=True)
    B.stab_engine_counters(sim.ctx, reset=True)
    B.stab_profile(sim.ctx, 0)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)

    def run_steps(profiled):
        evs = []
        for s in range(W, W + K):
            flush.fill_(s)                   # L2 flush between timed steps (outside the events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step(s)
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    # timed region: the library replays each step's launch sequence as a CUDA graph
    t_wall0 = time.perf_counter()
    step_ms = run_steps(False)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    sim.sync()
    launches = B.stab_launch_count(sim.ctx, reset=True)
    counters = B.stab_engine_counters(sim.ctx, reset=True)
    value, t_dev = aggregate(sum(step_ms) / 1e3, ops_per_step, K, world, dist, sim.device)
    recs = B.records_to_numpy(rec)
    # per-kernel durations: CUDA events around every launch, over K more steps
    # on the same inputs (per-launch events turn graph replay off, so they are
    # kept out of the timed steps); the records must come out the same
    B.stab_profile(sim.ctx, 0xFF)
    for k in sorted(B.KERNEL_NAMES):
        B.stab_profile_read(sim.ctx, k, reset=True)
    step_ms_prof = run_steps(True)
    sim.sync()
    B.stab_profile(sim.ctx, 0)
    B.stab_launch_count(sim.ctx, reset=True)
    counters_prof = B.stab_engine_counters(sim.ctx, reset=True)
    kstats = {B.KERNEL_NAMES[k]: B.stab_profile_read(sim.ctx, k, reset=True) for k in sorted(B.KERNEL_NAMES)}
    if not np.array_equal(B.records_to_numpy(rec), recs):
        raise AssertionError("graph replay and plain launches gave different records")


    # ---- e2e: host buffers through the C ABI, copies inside the timed region
    pin_c = torch.from_numpy(coins.view(np.int64)).pin_memory()
    pin_n = torch.from_numpy(noise.view(np.int32)).pin_memory()
    cnp, nnp = pin_c.numpy().view(np.uint64), pin_n.numpy().view(np.uint32)
    host_rec = np.zeros((1, circ.record_words), np.uint64)
    import ctypes
    lib = B.lib()
    e2e_t = []
    rec_words = circ.record_words            # a scan of the op list: kept out of the timed call
    for s in range(0 if args.no_e2e else min(K, 3) + 1):
        argv = (sim.ctx, cid, 1, cnp[s].ctypes.data_as(ctypes.c_void_p), cnp.shape[1],
                nnp[s].ctypes.data_as(ctypes.c_void_p), nnp.shape[1],
                host_rec.ctypes.data_as(ctypes.c_void_p), rec_words, B.ENGINE_LAYERED)
        flush.fill_(s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = lib.stab_sample_host(*argv)
        dt = time.perf_counter() - t0
        B._check(rc)
        if s:
            e2e_t.append(dt)
        if not np.array_equal(host_rec[0], recs[s]):
            raise AssertionError("host-buffer call gave a different record than the device-buffer call")
    e2e_val = ops_per_step * world / float(np.mean(e2e_t)) if e2e_t else None

    # ---- roofline of the dominant kernel, against HBM or L2 by working set
    dom = max(kstats, key=lambda k: kstats[k]["total_ms"])
    ds = kstats[dom]
    hbm, src = peaks()
    l2 = l2_sweep(sim, B, torch)
    l2_gbs, l2_size = l2["l2_gbs"], min(l2["l2_cache_bytes"] or 0, l2["l2_effective_bytes"])
    qm_b, rm_b = tableau_bytes(circ.n)
    # one launch's working set: a gate run reads and writes the column-packed
    # copy and writes the row-packed stabilizer half; the random-measurement
    # kernel works on the row-packed copy and the layer's measured columns
    max_layer = int(info.get("max_layer_meas", 0))
    ws = {"k_gate_run": qm_b + rm_b // 2,
          "k_meas_rand": rm_b + 4 * max_layer * 2 * ((circ.n + 31) // 32)}
    row_bytes = 2 * circ.n / 8.0          # a tableau row (x and z) or column (2n rows), in bytes
    alg = ds["alg_bytes"]
    model = "library model" if alg > 0 else None
    if dom == "k_meas_rand" and counters_prof.get("wave_ops"):
        # each needed bit read once and written once: per random measurement
        # its column (which rows anticommute), the pivot row once, its copy into
        # the destabilizer and the new stabilizer row (4 row/column transfers);
        # per rowsum the row read and written (2)
        alg = (4 * counters_prof["wave_ops"] + 2 * counters_prof["sum_A"]) * row_bytes
        model = "(4 x random measurements + 2 x rowsums) x 2n/8 bytes"
    if ds["launches"] and alg > 0:
        ach = alg / (ds["total_ms"] / 1e3) / 1e9
        tr, tr_tag = ncu_traffic(dom)
        bnd = roof_bound(ws.get(dom, float("inf")), l2_size)
        pk = l2_gbs if bnd == "l2" else hbm
        roof = {"bound": bnd, "kernel": dom, "achieved": ach, "peak": pk, "unit": "GB/s",
                "frac": ach / pk, "peak_source": "measured (L2 copy probe, this run)" if bnd == "l2" else src,
                "frac_hbm": ach / hbm, "frac_l2": ach / l2_gbs, "working_set_bytes": ws.get(dom),
                "traffic": tr, "traffic_source": tr_tag,
                "alg_bytes_per_launch": alg / ds["launches"], "alg_model": model,
                "avg_launch_us": 1e3 * ds["total_ms"] / ds["launches"]}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": hbm, "unit": "GB/s",
                "frac": None, "peak_source": src, "traffic": None,
                "note": "dominant kernel has no algorithmic-byte model"}
    gr = kstats.get("k_gate_run")
    gate_roof = None
    if gr and gr["launches"]:
        ach = gr["alg_bytes"] / (gr["total_ms"] / 1e3) / 1e9
        tr, tr_tag = ncu_traffic("k_gate_run")
        bnd = roof_bound(ws["k_gate_run"], l2_size)
        pk = l2_gbs if bnd == "l2" else hbm
        gate_roof = {"kernel": "k_gate_run", "bound": bnd, "achieved": ach, "peak": pk, "frac": ach / pk,
                     "frac_hbm": ach / hbm, "frac_l2": ach / l2_gbs, "working_set_bytes": ws["k_gate_run"],
                     "unit": "GB/s", "launches": gr["launches"],
                     "alg_bytes_per_launch": gr["alg_bytes"] / gr["launches"],
                     "traffic": tr, "traffic_source": tr_tag,
                     "avg_launch_us": 1e3 * gr["total_ms"] / gr["launches"]}

    line = {
        "metric": METRIC, "value": value, "unit": "ops/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": 1e3 * t_dev / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"rotated surface-code Z-memory d={d}, {d} rounds, "
                               f"depolarizing p={p}, single shot per step",
                   "d": d, "n": circ.n, "ops_per_step": ops_per_step,
                   "noise_ops_per_step": circ.n_noise, "layers": info["n_layers"],
                   "engine": "layered", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between timed steps (512 MiB write)",
                   "streams": "device-resident coin/noise buffers"},
        "e2e": {"value": e2e_val, "unit": "ops/s",
                "h2d_bytes_per_step": int(coins[0].nbytes + noise[0].nbytes),
                "d2h_bytes_per_step": int(circ.record_words * 8)},
        "rates": {"gates_per_s": n_gates * world * K / t_dev, "measurements_per_s": n_meas_ops * world * K / t_dev,
                  "m_per_s": n_m_ops * world * K / t_dev, "r_per_s": n_r_ops * world * K / t_dev,
                  "gate_plus_m_ops_per_s": (n_gates + n_m_ops) * world * K / t_dev,
                  "shots_per_s": world * K / t_dev,
                  "ops_per_step": {"gates": n_gates, "M": n_m_ops, "R": n_r_ops},
                  "note": "gates: H/S/X/Y/Z/CX/CZ/SWAP ops; measurements: M and R ops (both Z "
                          "measurements); an R that directly follows an M on its qubit is folded into "
                          "that M (deterministic, an X when the outcome is 1), so gate_plus_m_ops_per_s "
                          "is the rate without resets"},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "l2": l2,
        "roofline_gate_run": gate_roof,
        "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"]} for k, v in kstats.items()},
        "engine_counters_per_step": {k: v / K for k, v in counters_prof.items()},
        "kernel_timing": "CUDA events around each launch over K further steps (plain launches, "
                         f"{float(np.mean(step_ms_prof)):.3f} ms per step); the timed steps replay CUDA graphs",
        "wall_s_timed": t_wall,
    }
    stage("timed steps done")
    if rank == 0 and not args.no_cpu:
        v, desc, _ = oracle_ops_per_s(circ, coins[0], noise[0], budget_s=15.0)
        line["cpu_baseline"] = {"value": v, "unit": "ops/s", "cores": 1, "kind": "oracle",
                                "sample": desc}
    if rank == 0 and not args.no_extras:
        stage("batched")
        try:
            line["batched"] = batched_vs_plain(sim, B, torch)
        except Exception as ex:       # report, do not hide
            line["batched"] = {"error": repr(ex)}
        if not args.no_cpu:
            try:
                line["batched"]["cpu_baseline"] = oracle_batched()
            except Exception as ex:
                line["batched"]["cpu_baseline"] = {"error": repr(ex)}
    if rank == 0 and not args.no_extras and not args.no_configs:
        stage("configs")
        try:
            line["configs"] = config_suite(sim, B, torch, flush, cpu=not args.no_cpu)
        except Exception as ex:       # report, do not hide
            line["configs"] = {"error": repr(ex)}
    if rank == 0 and (args.serve or world == 1) and not args.no_serve and not args.no_extras:
        from paper_2507_03092_gb300 import serve_trace
        circs = serve_trace.compile_circuits(sim)
        stage("serve replay")
        line["serve"] = serve_trace.replay(sim, B, torch, circs=circs)
        stage("serve capacity")
        try:
            sat = serve_trace.saturated(sim, B, torch, circs=circs)
            pl = serve_trace.plain(sim, B, torch, circs=circs)
            line["serve"]["saturated"] = sat
            line["serve"]["capacity_shots_per_s"] = sat["capacity_shots_per_s"]
            line["serve"]["plain"] = pl
            line["serve"]["plain_shots_per_s"] = pl["plain_shots_per_s"]
            if sat["capacity_shots_per_s"]:
                line["serve"]["served_over_plain"] = sat["capacity_shots_per_s"] / pl["plain_shots_per_s"]
        except Exception as ex:       # report, do not hide
            line["serve"]["capacity_error"] = repr(ex)
    sim.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
