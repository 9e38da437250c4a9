"""stab_sample_batch_noalloc: the batch launch for callers that cannot allocate
device memory when they call (every device allocation is owned by a host
framework's pool, or cudaMalloc's implicit synchronisation is unaffordable in
their loop).  Its job table and work counter live in a fixed array compiled
into the library, so its records must equal those of stab_sample_batch, which
allocates that scratch with cudaMalloc.  Two calls in a row check that the
shared array's leftover contents (the previous call's jobs and counter) do
not leak into the next call."""
import numpy as np
import pytest

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


def _groups(sim, specs, seed):
    """Job groups with device coin/noise buffers; returns (groups, records, keep)."""
    groups, recs, keep = [], [], []
    for circ, shots in specs:
        cid = sim.compile(circ)
        coins, noise = S.streams_for(circ, seed, range(shots))
        dc, dn = sim.to_dev(coins), sim.to_dev(noise)
        rec = sim.record_buffer(shots, circ.record_words)
        g = B.JobGroup()
        g.circuit_id, g.shots = cid, shots
        g.streams = B.make_streams(B.STREAM_BUFFER, coins=dc, noise=dn)
        g.d_record, g.record_words = rec.data_ptr(), circ.record_words
        groups.append(g)
        recs.append(rec)
        keep += [dc, dn]
    return groups, recs, keep


def test_noalloc_batch_matches_allocating_batch_twice(sim):
    T = {"T1": 100e-6, "T2": 80e-6, "t1q": 50e-9, "t2q": 300e-9, "tm": 1e-6}
    specs = [(C.surface_code_memory(3, p=0.01), 200),
             (C.surface_code_memory(5, t1t2=T), 60),
             (C.random_small_circuit(40, 300, seed=4), 25)]
    ref_groups, ref_recs, keep = _groups(sim, specs, seed=11)
    B.stab_sample_batch(sim.ctx, ref_groups)
    sim.sync()
    want = [B.records_to_numpy(r) for r in ref_recs]
    for call in range(2):
        groups, recs, keep2 = _groups(sim, specs, seed=11)
        B.stab_sample_batch_noalloc(sim.ctx, groups)
        sim.sync()
        for w, r in zip(want, recs):
            assert np.array_equal(B.records_to_numpy(r), w), f"call {call}"


def test_noalloc_rejects_batches_beyond_its_fixed_size(sim):
    circ = C.ghz(4)
    cid = sim.compile(circ)
    # sized for every requested shot, so that a regression of the host-side
    # limit check fails on the assertion below instead of writing past a buffer
    rec = sim.record_buffer(8193, circ.record_words)
    g = B.JobGroup()
    g.circuit_id, g.shots = cid, 8193
    g.streams = B.make_streams(B.STREAM_SEEDED, seed=1)
    g.d_record, g.record_words = rec.data_ptr(), circ.record_words
    with pytest.raises(B.StabError) as e:
        B.stab_sample_batch_noalloc(sim.ctx, [g])
    assert e.value.code == B.ERR_UNSUPPORTED and "8192" in str(e.value)
