"""CPU oracle: plain Aaronson-Gottesman (CHP) tableau simulator (``chp.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline / reference legs may import this package.  It
shares no code with the CUDA path (``paper_2507_03092_gb300``) and never
imports it; both sides read the same seeded inputs from
``paper_2507_03092_gb300.circuit`` / ``.streams``, which hold no simulation
arithmetic.

Every function here only marshals arguments; the arithmetic is in ``chp.c``,
whose header cites the paper passages it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chp.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "bad argument", -2: "out of memory", -4: "stream too short",
          -10: "odd phase in rowsum", -11: "deterministic product is not +-Z_a (or +-P)"}


class OracleError(RuntimeError):
    pass


class Stats(ctypes.Structure):
    _fields_ = [("n_meas_random", ctypes.c_uint64), ("n_meas_det", ctypes.c_uint64),
                ("sum_A", ctypes.c_uint64), ("sum_K", ctypes.c_uint64),
                ("n_gates", ctypes.c_uint64), ("n_noise_events", ctypes.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile chp.c with gcc into oracle/_build/liboracle.so (host code only)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The oracle library: built from chp.c, or the prebuilt library named by
    the ORACLE_LIB environment variable (the planted-mistake tests point it at
    mutated copies of chp.c)."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
            P, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
            L.chp_new.restype = P
            L.chp_new.argtypes = [u32]
            L.chp_free.argtypes = [P]
            L.chp_reset.argtypes = [P]
            L.chp_words.restype = u32
            L.chp_words.argtypes = [P]
            L.chp_get.argtypes = [P, P, P, P]
            L.chp_set.argtypes = [P, P, P, P]
            L.chp_g.restype = ctypes.c_int
            L.chp_g.argtypes = [ctypes.c_int] * 4
            L.chp_run.restype = ctypes.c_int
            L.chp_run.argtypes = [P, P, sz, P, sz, P, sz, P, sz, P, sz, ctypes.POINTER(Stats)]
            L.chp_commute.restype = ctypes.c_int
            L.chp_commute.argtypes = [P, P, P, sz, P]
            L.chp_sample.restype = ctypes.c_int
            L.chp_sample.argtypes = [u32, P, sz, P, sz, u64, P, sz, P, sz, P, sz,
                                     ctypes.c_int, ctypes.POINTER(Stats)]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


def g(x1, z1, x2, z2) -> int:
    return int(lib().chp_g(int(x1), int(z1), int(x2), int(z2)))


class Tableau:
    """One CHP state; ``run`` applies a circuit with its own streams."""

    def __init__(self, n: int):
        self.n = n
        self._h = lib().chp_new(n)
        if not self._h:
            raise MemoryError("chp_new failed")
        self.W = int(lib().chp_words(self._h))
        self.stats = Stats()

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.chp_free(h)

    def reset(self):
        lib().chp_reset(self._h)

    def run(self, circuit, coins=None, noise=None) -> np.ndarray:
        """Apply ``circuit`` (coins: uint64[words], noise: uint32[words]);
        returns the uint64 record of its M ops."""
        if circuit.n != self.n:
            raise ValueError("qubit count mismatch")
        ops = np.ascontiguousarray(circuit.ops)
        params = np.ascontiguousarray(circuit.params, dtype=np.float64)
        coins = np.zeros(circuit.coin_words, np.uint64) if coins is None else \
            np.ascontiguousarray(coins, dtype=np.uint64).ravel()
        noise = np.zeros(circuit.noise_words, np.uint32) if noise is None else \
            np.ascontiguousarray(noise, dtype=np.uint32).ravel()
        rec = np.zeros(circuit.record_words, np.uint64)
        rc = lib().chp_run(self._h, _ptr(ops), len(ops), _ptr(params), len(params),
                           _ptr(coins), coins.size, _ptr(noise), noise.size,
                           _ptr(rec), rec.size, ctypes.byref(self.stats))
        if rc:
            raise OracleError(ERRORS.get(rc, str(rc)))
        return rec

    def get(self):
        """(x, z, r): uint64 [2n, W], uint64 [2n, W], uint8 [2n]."""
        x = np.zeros((2 * self.n, self.W), np.uint64)
        z = np.zeros((2 * self.n, self.W), np.uint64)
        r = np.zeros(2 * self.n, np.uint8)
        lib().chp_get(self._h, _ptr(x), _ptr(z), _ptr(r))
        return x, z, r

    def commute(self, px, pz) -> np.ndarray:
        """Anticommutation of m Paulis (px, pz: uint64 [m, W]) with every row:
        uint64 [m, ceil(2n/64)], bit i = row i anticommutes."""
        px = np.ascontiguousarray(px, np.uint64).reshape(-1, self.W)
        pz = np.ascontiguousarray(pz, np.uint64).reshape(-1, self.W)
        m = px.shape[0]
        out = np.zeros((m, (2 * self.n + 63) // 64), np.uint64)
        if m:
            lib().chp_commute(self._h, _ptr(px), _ptr(pz), m, _ptr(out))
        return out

    def set(self, x, z, r):
        x = np.ascontiguousarray(x, np.uint64)
        z = np.ascontiguousarray(z, np.uint64)
        r = np.ascontiguousarray(r, np.uint8)
        lib().chp_set(self._h, _ptr(x), _ptr(z), _ptr(r))


def run(circuit, coins=None, noise=None, return_tableau=False):
    t = Tableau(circuit.n)
    rec = t.run(circuit, coins, noise)
    if return_tableau:
        return rec, t.get(), t.stats.as_dict()
    return rec


def sample(circuit, coins: np.ndarray, noise: np.ndarray, threads: int = 1):
    """Independent shots from |0..0>: coins uint64 [S, cw], noise uint32 [S, nw].
    Returns (records uint64 [S, rw], stats dict)."""
    coins = np.ascontiguousarray(coins, np.uint64)
    noise = np.ascontiguousarray(noise, np.uint32)
    S = coins.shape[0]
    if noise.shape[0] != S:
        raise ValueError("stream shot counts differ")
    rec = np.zeros((S, circuit.record_words), np.uint64)
    ops = np.ascontiguousarray(circuit.ops)
    params = np.ascontiguousarray(circuit.params, dtype=np.float64)
    st = Stats()
    rc = lib().chp_sample(circuit.n, _ptr(ops), len(ops), _ptr(params), len(params), S,
                          _ptr(coins), coins.shape[1], _ptr(noise), noise.shape[1],
                          _ptr(rec), rec.shape[1], int(threads), ctypes.byref(st))
    if rc:
        raise OracleError(ERRORS.get(rc, str(rc)))
    return rec, st.as_dict()


def record_bits(rec: np.ndarray, n_bits: int) -> np.ndarray:
    """Unpack uint64 record words (last axis) into n_bits uint8 bits."""
    rec = np.asarray(rec, np.uint64)
    b = np.unpackbits(rec.view(np.uint8).reshape(rec.shape[:-1] + (-1,)),
                      axis=-1, bitorder="little")
    return b[..., :n_bits]
