"""Host-side checks of the layered engine's packed gate layers (no GPU).

The slice kernel keeps column j of a 32-row slice in shared-memory slot
gate_slot(j), and the compiler stores each gate layer's items in an order
chosen for the kernel's shared-memory banks, with their operands' slots.  A
small host program (tests/layout_check.cpp, built here with the library's
compiler from the same compile.cpp) checks that gate_slot permutes every
aligned block of 16 columns and is its own inverse, and that every gate
layer's packed items are its items reordered, then reports each layer's
shared-memory wavefronts.  On the d = 71 surface-code circuit the packed order
must come close to one wavefront per 16 operands and stay well below the
circuit order with unswizzled slots (whose CX operands run in steps of two and
so fill half the bank pairs)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2507_03092_gb300 import build as BLD
from paper_2507_03092_gb300 import circuit as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    try:
        cc = BLD.nvcc()
    except Exception as ex:          # no CUDA toolkit on this machine
        pytest.skip("nvcc not found: %r" % ex)
    if not cc or not shutil.which(cc):
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("layout") / "layout_check")
    cmd = [cc] + BLD.GENCODE + ["-O2", "-std=c++17", "--expt-relaxed-constexpr", "-I",
                                os.path.join(ROOT, "include"), "-x", "cu",
                                os.path.join(ROOT, "tests", "layout_check.cpp"),
                                os.path.join(ROOT, "paper_2507_03092_gb300", "csrc", "compile.cpp"),
                                "-o", out, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return out


def _run(checker, circ, tmp_path):
    ops, params = tmp_path / "ops.bin", tmp_path / "params.bin"
    np.ascontiguousarray(circ.ops, dtype=C.OP_DTYPE).tofile(ops)
    np.ascontiguousarray(circ.params, dtype=np.float64).reshape(-1, 3).tofile(params)
    r = subprocess.run([checker, str(ops), str(params), str(circ.n)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = r.stdout.splitlines()
    assert lines[0] == "slot ok"
    layers = []
    for ln in lines[1:]:
        _, l, count, two, now, ident, ideal = ln.split()
        layers.append((int(l), int(count), two == "1", int(now), int(ident), int(ideal)))
    return layers


def test_d71_gate_layers_reach_the_banks(checker, tmp_path):
    layers = _run(checker, C.surface_code_memory(71, p=1e-3), tmp_path)
    assert len(layers) == 71 * 6          # H, four CX steps, H per round
    now = sum(x[3] for x in layers)
    ident = sum(x[4] for x in layers)
    ideal = sum(x[5] for x in layers)
    assert now <= 1.12 * ideal, (now, ideal)
    assert now <= 0.7 * ident, (now, ident)
    for l, count, two, n_, i_, id_ in layers:
        assert n_ <= 1.25 * id_, (l, count, two, n_, id_)


@pytest.mark.parametrize("n", [1, 15, 17, 100, 333])
def test_small_and_ragged_circuits_pack_every_item(checker, tmp_path, n):
    # random layers of one- and two-qubit gates with noise on n qubits: the
    # checker exits non-zero if a packed layer is not its items reordered
    circ = C.random_small_circuit(n, 40 * n + 10, seed=n)
    assert _run(checker, circ, tmp_path) is not None
