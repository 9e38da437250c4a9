"""Write the golden fixtures of tests/golden/ from the CPU oracle only.

Every fixture is the oracle's output on seeded synthetic inputs; nothing here
imports or runs the CUDA path.  Records are stored as SHA-256 digests of their
little-endian uint64 words plus summary counts, so the GPU tests can check
every outcome bit without large fixtures.

d71_noisy_seed0.json: the full d=71, 71-round rotated surface-code Z-memory
circuit with DEPOLARIZE1/2(1e-3) after every H/CNOT, shot 0 of seed 0 (the
benchmark's first warm-up shot).

d71_noiseless_seed{0,1}.json: the same circuit without noise (the first half
of the "noiseless then depolarizing" d=71 workload), shot 0 of seeds 0 and 1:
the round-1 X-ancilla outcomes follow the coins, everything after is fixed by
them.

serve_largest.json: the largest requests of the serving workload (d uniform
odd in 3..31, shots uniform 1..256, DEPOLARIZE1/2(1e-3)): d=31 with 256 shots
and d=29 with 200 shots, streams keyed by (request seed, shot) as the serving
loop's seeded mode keys them; one digest per shot.

    python tests/golden/make_golden.py [noisy|noiseless|serve|all]
    (noisy about 14 minutes on one core; noiseless about 14 minutes per seed,
    the two seeds run in parallel; serve about 5 minutes on 8 cores)
"""
import hashlib
import json
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2507_03092_gb300 import circuit as C  # noqa: E402
from paper_2507_03092_gb300 import streams as S  # noqa: E402

# (d, shots, request seed) of the largest serving requests checked at full size
SERVE_LARGEST = ((31, 256, 9031), (29, 200, 9029))


def digest(words: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(words, "<u8").tobytes()).hexdigest()


def d71_record(p: float, seed: int) -> dict:
    circ = C.surface_code_memory(71, p=p)
    coins, noise = S.streams_for(circ, seed, [0])
    t0 = time.time()
    rec = oracle.run(circ, coins[0], noise[0])
    bits = oracle.record_bits(rec, circ.n_meas)
    det = [int(np.bitwise_xor.reduce(bits[d])) for d in circ.meta["detectors"]]
    return {
        "circuit": f"surface_code_memory(71, p={p:g})" if p else "surface_code_memory(71)",
        "seed": seed, "shot": 0,
        "n_meas": circ.n_meas, "record_words": int(rec.size),
        "record_sha256": digest(rec),
        "ones": int(bits.sum()), "detectors_fired": int(sum(det)),
        "oracle_seconds": round(time.time() - t0, 1),
    }


def write(name: str, obj: dict) -> None:
    with open(os.path.join(HERE, name), "w") as fh:
        json.dump(obj, fh, indent=1)
    print(name, {k: v for k, v in obj.items() if k != "requests"})


def noisy():
    write("d71_noisy_seed0.json", d71_record(1e-3, 0))


def noiseless():
    with ProcessPoolExecutor(2) as ex:
        outs = list(ex.map(d71_record, [0.0, 0.0], [0, 1]))
    for seed, out in zip((0, 1), outs):
        write(f"d71_noiseless_seed{seed}.json", out)


def serve():
    threads = os.cpu_count() or 1
    reqs = []
    t0 = time.time()
    for d, shots, seed in SERVE_LARGEST:
        circ = C.surface_code_memory(d, p=1e-3)
        coins, noise = S.streams_for(circ, seed, range(shots))
        rec, _ = oracle.sample(circ, coins, noise, threads=threads)
        reqs.append({"d": d, "shots": shots, "seed": seed, "record_words": int(rec.shape[1]),
                     "n_meas": circ.n_meas,
                     "shot_sha256": [digest(rec[s])[:32] for s in range(shots)],
                     "ones": int(oracle.record_bits(rec, circ.n_meas).sum())})
    write("serve_largest.json", {"circuit": "surface_code_memory(d, p=1e-3)",
                                 "streams": "SplitMix64 keyed by (request seed, shot)",
                                 "requests": reqs, "oracle_seconds": round(time.time() - t0, 1),
                                 "threads": threads})


def main():
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("noisy", "all"):
        noisy()
    if what in ("noiseless", "all"):
        noiseless()
    if what in ("serve", "all"):
        serve()


if __name__ == "__main__":
    main()
