"""Write the golden fixtures of tests/golden/ from the CPU oracle only.

d71_noisy_seed0.json: the full d=71, 71-round rotated surface-code Z-memory
circuit with DEPOLARIZE1/2(1e-3) after every H/CNOT, shot 0 of seed 0 (the
benchmark's first warm-up shot).  The oracle's record is stored as a SHA-256
digest of its little-endian uint64 words plus summary counts, so the GPU test
can check all 362 881 outcome bits without a large fixture.

    python tests/golden/make_golden.py      (about 5 minutes, one core)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2507_03092_gb300 import circuit as C  # noqa: E402
from paper_2507_03092_gb300 import streams as S  # noqa: E402


def main():
    circ = C.surface_code_memory(71, p=1e-3)
    coins, noise = S.streams_for(circ, 0, [0])
    t0 = time.time()
    rec = oracle.run(circ, coins[0], noise[0])
    bits = oracle.record_bits(rec, circ.n_meas)
    det = [int(np.bitwise_xor.reduce(bits[d])) for d in circ.meta["detectors"]]
    out = {
        "circuit": "surface_code_memory(71, p=1e-3)", "seed": 0, "shot": 0,
        "n_meas": circ.n_meas, "record_words": int(rec.size),
        "record_sha256": hashlib.sha256(np.ascontiguousarray(rec, "<u8").tobytes()).hexdigest(),
        "ones": int(bits.sum()), "detectors_fired": int(sum(det)),
        "oracle_seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(HERE, "d71_noisy_seed0.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    main()
