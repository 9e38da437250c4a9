"""Pauli-product measurement (MPP) on both engines and the Pauli-vs-tableau
commutation kernel (stab_commute), against the CPU oracle on the same seeded
inputs.  The resident engine applies the direct rule; the layered engine the
Clifford conjugation of a Z measurement, whose tableau may hold a different
(equivalent) set of generators, so it is compared through records -- including
a suffix of random Pauli-product measurements that would expose any
difference in the stabilizer group -- and through the tableau invariants."""
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


def _both_engines(sim, circ, shots, seed):
    coins, noise = S.streams_for(circ, seed, range(shots))
    want, _ = oracle.sample(circ, coins, noise, threads=8)
    cid = sim.compile(circ)
    for eng in (B.ENGINE_RESIDENT, B.ENGINE_LAYERED):
        got = B.records_to_numpy(sim.sample(cid, circ, shots, coins, noise, engine=eng))
        sim.sync()
        assert np.array_equal(got, want), (circ.n, seed, eng)
    sim.release(cid)


def _random_mpp_suffix(n, count, seed, max_w=8):
    rng = np.random.default_rng(seed)
    b = C.Builder(n)
    for _ in range(count):
        k = int(rng.integers(1, min(n, max_w) + 1))
        qs = rng.choice(n, size=k, replace=False)
        b.mpp([(int(q), int(rng.integers(1, 4))) for q in qs])
    return b.build()


@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 64, 97])
def test_random_mpp_circuits_both_engines(sim, n):
    for seed in range(3):
        circ = C.random_small_circuit(n, 40 if n <= 8 else 4 * n, seed=seed + 31 * n, mpp=True)
        assert int(np.count_nonzero(circ.ops["kind"] == C.MPP)) > 0
        _both_engines(sim, circ, 24, seed)


def test_wide_products_up_to_64_factors(sim):
    n = 200
    for seed in range(2):
        base = C.random_clifford_layers(n, 6, seed=seed)
        suf = _random_mpp_suffix(n, 120, seed, max_w=64)
        circ = C.concat([base, suf])
        _both_engines(sim, circ, 8, seed)


def test_mpp_surface_code_both_engines(sim):
    for d, p in ((3, 1e-2), (5, 1e-2), (7, 5e-3), (15, 1e-3)):
        circ = C.surface_code_mpp(d, p=p)
        _both_engines(sim, circ, 32, d)


def test_mpp_surface_code_noiseless_detectors(sim):
    circ = C.surface_code_mpp(11)
    cid = sim.compile(circ)
    for eng in (B.ENGINE_RESIDENT, B.ENGINE_LAYERED):
        rec = B.records_to_numpy(sim.sample(cid, circ, 8, seed=3, engine=eng))
        sim.sync()
        bits = oracle.record_bits(rec, circ.n_meas)
        for det in circ.meta["detectors"]:
            assert not np.bitwise_xor.reduce(bits[:, det], axis=1).any()


def _symplectic_ok(x, z, n):
    W = x.shape[1]
    xb = np.unpackbits(x.view(np.uint8).reshape(2 * n, 8 * W), axis=1, bitorder="little")[:, :n].astype(np.int64)
    zb = np.unpackbits(z.view(np.uint8).reshape(2 * n, 8 * W), axis=1, bitorder="little")[:, :n].astype(np.int64)
    inner = (xb @ zb.T + zb @ xb.T) % 2
    J = np.zeros((2 * n, 2 * n), np.int64)
    J[np.arange(n), np.arange(n) + n] = 1
    J[np.arange(n) + n, np.arange(n)] = 1
    return np.array_equal(inner, J)


@pytest.mark.parametrize("n", [7, 40, 130])
def test_layered_tableau_after_mpp_is_equivalent(sim, n):
    """stab_apply_circuit (layered engine) on an MPP circuit: records equal
    the oracle's, the tableau keeps the CHP invariants, and a suffix of 200
    random Pauli-product measurements (run on top of that tableau) gives the
    oracle's records too."""
    circ = C.random_small_circuit(n, 3 * n + 30, seed=n, mpp=True)
    suf = _random_mpp_suffix(n, 200, n + 1)
    full = C.concat([circ, suf])
    coins, noise = S.streams_for(full, 9, range(4))
    want, _ = oracle.sample(full, coins, noise)
    cid, sid = sim.compile(circ), sim.compile(suf)
    B.stab_tableau_init(sim.ctx, n, 4)
    # the prefix consumes the first coin/noise words of each shot
    c1, n1 = S.streams_for(circ, 9, range(4))
    rec1 = sim.record_buffer(4, circ.record_words)
    B.stab_apply_circuit(sim.ctx, cid, B.make_streams(B.STREAM_BUFFER, coins=sim.to_dev(c1),
                                                      noise=sim.to_dev(n1)), rec1)
    sim.sync()
    w1, _ = oracle.sample(circ, c1, n1)
    assert np.array_equal(B.records_to_numpy(rec1), w1)
    for t in range(4):
        x, z, _ = B.stab_get_tableau(sim.ctx, t, n)
        assert _symplectic_ok(x, z, n)
    # suffix coins: the full circuit's coin bits after the prefix's
    nb = circ.n_coin
    bits = np.unpackbits(coins.view(np.uint8).reshape(4, -1), axis=1, bitorder="little")
    sb = bits[:, nb:nb + suf.n_coin]
    sb = np.pad(sb, ((0, 0), (0, 64 * suf.coin_words - sb.shape[1])))
    c2 = np.packbits(sb, axis=1, bitorder="little").view(np.uint64).reshape(4, suf.coin_words)
    rec2 = sim.record_buffer(4, suf.record_words)
    B.stab_apply_circuit(sim.ctx, sid, B.make_streams(B.STREAM_BUFFER, coins=sim.to_dev(c2),
                                                      noise=sim.to_dev(np.zeros((4, 1), np.uint32))), rec2)
    sim.sync()
    got = np.concatenate([oracle.record_bits(B.records_to_numpy(rec1), circ.n_meas),
                          oracle.record_bits(B.records_to_numpy(rec2), suf.n_meas)], axis=1)
    assert np.array_equal(got, oracle.record_bits(want, full.n_meas))


@pytest.mark.parametrize("n", [1, 31, 32, 33, 64, 65, 130, 257])
def test_commute_matches_oracle(sim, n):
    torch = pytest.importorskip("torch")
    circ = C.random_small_circuit(n, 6 * n + 20, seed=7 * n, noise=False)
    coins, noise = S.streams_for(circ, 5, [0, 1])
    _, otab, _ = oracle.run(circ, coins[1], noise[1], return_tableau=True)
    cid = sim.compile(circ)
    B.stab_tableau_init(sim.ctx, n, 2)
    rec = sim.record_buffer(2, circ.record_words)
    B.stab_apply_circuit(sim.ctx, cid, B.make_streams(B.STREAM_BUFFER, coins=sim.to_dev(coins),
                                                      noise=sim.to_dev(noise)), rec)
    sim.sync()
    for g, w in zip(B.stab_get_tableau(sim.ctx, 1, n), otab):     # same tableau as the oracle's
        assert np.array_equal(g, w)
    Wq = (n + 63) // 64
    rng = np.random.default_rng(n)
    for m in (1, 37, 300):
        px = rng.integers(0, 2 ** 63, size=(m, Wq), dtype=np.uint64) * np.uint64(2) + \
            rng.integers(0, 2, size=(m, Wq), dtype=np.uint64)        # bits >= n are ignored
        pz = rng.integers(0, 2 ** 63, size=(m, Wq), dtype=np.uint64) * np.uint64(2)
        pz[::3] = 0                                                  # pure X strings
        px[1::5] = 0                                                 # pure Z strings
        d_px = torch.from_numpy(px.view(np.int64)).cuda()
        d_pz = torch.from_numpy(pz.view(np.int64)).cuda()
        out = torch.full((m, 2 * Wq), -1, dtype=torch.int64, device="cuda")
        B.stab_commute(sim.ctx, 1, d_px, d_pz, m, out)
        got = out.cpu().numpy().view(np.uint64)
        t = oracle.Tableau(n)
        t.set(*otab)
        want = t.commute(px, pz)
        wb = np.unpackbits(want.view(np.uint8).reshape(m, -1), axis=1, bitorder="little")[:, :2 * n]
        gd = np.unpackbits(got[:, :Wq].view(np.uint8).reshape(m, -1), axis=1, bitorder="little")
        gs = np.unpackbits(got[:, Wq:].view(np.uint8).reshape(m, -1), axis=1, bitorder="little")
        assert np.array_equal(gd[:, :n], wb[:, :n])
        assert np.array_equal(gs[:, :n], wb[:, n:])
        assert not gd[:, n:].any() and not gs[:, n:].any()          # padding bits zero
    B.stab_commute(sim.ctx, 1, None, None, 0, None)                   # m = 0: nothing to do


def test_commute_argument_errors(sim):
    B.stab_tableau_init(sim.ctx, 10, 1)
    with pytest.raises(B.StabError) as e:
        B.stab_commute(sim.ctx, 1, None, None, 1, None)
    assert e.value.code == B.ERR_ARG


@pytest.mark.parametrize("ops", [
    [(C.MPP, 2, 0), (C.PAULI, 0, 3)],
    [(C.MPP, 2, 0), (C.PAULI, 0, 3), (C.PAULI, 0, 1)],
    [(C.MPP, 1, 0), (C.PAULI, 0, 4)],
    [(C.MPP, 1, 0), (C.H, 0, 0)],
    [(C.MPP, 0, 0), (C.H, 0, 0)],
    [(C.PAULI, 0, 1)],
    [(C.MPP, 1, 0), (C.PAULI, 2, 1)],
])
def test_bad_mpp_rejected_at_compile(sim, ops):
    b = C.Builder(2)
    for k, q0, q1 in ops:
        b.op(k, q0, q1)
    with pytest.raises(B.StabError) as e:
        sim.compile(b.build())
    assert e.value.code == B.ERR_ARG
