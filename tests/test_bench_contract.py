"""bench.py's command-line contract on the host: the reference arm (the CPU
oracle) prints one JSON line with the keys the contract names, ranks other
than 0 print nothing, and the GPU arm fails loudly where there is no GPU
instead of falling back to the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--d", "3", "--steps", "2", "--warmup", "3", "--ref-step-s", "0.05"]


def _bench(args, env=None, timeout=300):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, env=e, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _bench(["--impl", "reference"] + SMALL)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "ops/s" and d["higher_is_better"] is True
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 3, 1)
    assert d["value"] > 0 and d["config"]["d"] == 3 and d["config"]["n"] == 17
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert (e2e["value"], e2e["unit"]) == (d["value"], d["unit"])
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    r = _bench(["--impl", "reference"] + SMALL, env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_gpu_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _bench(["--steps", "1", "--warmup", "3", "--no-extras", "--no-cpu", "--no-e2e"])
    assert r.returncode != 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_batched_oracle_baseline_keys():
    import bench
    r = bench.oracle_batched(shots=256, per_d=4, cores=2)
    assert r["kind"] == "oracle" and r["cores"] == 2
    assert r["one_core_shots_per_s"] > 0 and r["all_cores_shots_per_s"] > 0
    assert "20 shots" in r["sample"]
