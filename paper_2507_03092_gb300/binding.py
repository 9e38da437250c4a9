"""ctypes binding to ``libstab.so`` (the C ABI in ``include/stab.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  Functions keep the C names (``stab_create``, ``stab_compile``,
``stab_tableau_init``, ``stab_apply_circuit``, ``stab_sample``, ...) and raise
``StabError`` on a non-zero status.  Device buffers are passed as torch CUDA
tensors (PyTorch is used only for device memory and streams).  There is no
CPU fallback: if the library is missing the import of this module's functions
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import circuit as C

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libstab.so")

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STREAM_SHORT = -1, -2, -3, -4
ERR_TIMEOUT, ERR_BUSY, ERR_INTERNAL, ERR_NOT_FOUND, ERR_UNSUPPORTED = -5, -6, -7, -8, -9
STREAM_BUFFER, STREAM_SEEDED = 0, 1
ENGINE_AUTO, ENGINE_LAYERED, ENGINE_RESIDENT = 0, 1, 2


class StabError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Streams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("rsv", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("shot_offset", ctypes.c_uint64),
                ("coins", ctypes.c_void_p), ("coin_words", ctypes.c_uint64),
                ("noise", ctypes.c_void_p), ("noise_words", ctypes.c_uint64)]


class CircuitInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("n_layers", ctypes.c_uint32),
                ("n_ops", ctypes.c_uint64), ("n_gates", ctypes.c_uint64),
                ("n_meas", ctypes.c_uint64), ("n_coin", ctypes.c_uint64),
                ("n_noise_words", ctypes.c_uint64), ("record_words", ctypes.c_uint64),
                ("coin_words", ctypes.c_uint64), ("n_gate_layers", ctypes.c_uint32),
                ("n_meas_layers", ctypes.c_uint32), ("n_gate_runs", ctypes.c_uint32),
                ("max_layer_meas", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class JobGroup(ctypes.Structure):
    _fields_ = [("circuit_id", ctypes.c_uint64), ("shots", ctypes.c_uint32),
                ("rsv", ctypes.c_uint32), ("streams", Streams),
                ("d_record", ctypes.c_void_p), ("record_words", ctypes.c_uint64)]


class Tune(ctypes.Structure):
    _fields_ = [("group_threads", ctypes.c_uint32), ("tableaux_per_cta", ctypes.c_uint32),
                ("words_per_thread", ctypes.c_uint32), ("rsv", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_[:3]}


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double)]

    def as_dict(self):
        return {"launches": int(self.launches), "total_ms": float(self.total_ms),
                "alg_bytes": float(self.alg_bytes)}


KERNEL_GATE_RUN, KERNEL_MEAS_DET, KERNEL_MEAS_RAND, KERNEL_OTHER, KERNEL_RESIDENT, KERNEL_COMMUTE = range(6)
KERNEL_NAMES = {KERNEL_GATE_RUN: "k_gate_run", KERNEL_MEAS_DET: "k_meas_det",
                KERNEL_MEAS_RAND: "k_meas_rand", KERNEL_OTHER: "other",
                KERNEL_RESIDENT: "k_resident", KERNEL_COMMUTE: "k_commute"}


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("n_streams", ctypes.c_uint32), ("max_batch_requests", ctypes.c_uint32),
                ("rsv", ctypes.c_uint32)]


class RequestStatus(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("shots", ctypes.c_uint32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


_lib = None
_lock = threading.Lock()

P, U32, U64, SZ, I32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
PP = ctypes.POINTER(ctypes.c_void_p)
PU64 = ctypes.POINTER(ctypes.c_uint64)

_SIGS = {
    "stab_create": (I32, [PP, I32, P]),
    "stab_destroy": (None, [P]),
    "stab_set_stream": (I32, [P, P]),
    "stab_last_error": (ctypes.c_char_p, []),
    "stab_sync": (I32, [P]),
    "stab_compile": (I32, [P, U32, P, SZ, P, SZ, PU64]),
    "stab_circuit_info_get": (I32, [P, U64, ctypes.POINTER(CircuitInfo)]),
    "stab_compile_info": (I32, [U32, P, SZ, P, SZ, ctypes.POINTER(CircuitInfo)]),
    "stab_release_circuit": (I32, [P, U64]),
    "stab_tableau_init": (I32, [P, U32, U32]),
    "stab_apply_circuit": (I32, [P, U64, ctypes.POINTER(Streams), P, U64]),
    "stab_get_tableau": (I32, [P, U32, P, P, P]),
    "stab_set_tableau": (I32, [P, U32, P, P, P]),
    "stab_commute": (I32, [P, U32, P, P, SZ, P]),
    "stab_sample": (I32, [P, U64, U32, ctypes.POINTER(Streams), P, U64, U32]),
    "stab_sample_host": (I32, [P, U64, U32, P, U64, P, U64, P, U64, U32]),
    "stab_sample_batch": (I32, [P, ctypes.POINTER(JobGroup), SZ]),
    "stab_sample_batch_noalloc": (I32, [P, ctypes.POINTER(JobGroup), SZ]),
    "stab_autotune": (I32, [P, PU64, SZ, U32]),
    "stab_get_tune": (I32, [P, U32, ctypes.POINTER(Tune)]),
    "stab_set_tune": (I32, [P, U32, ctypes.POINTER(Tune)]),
    "stab_serve_start": (I32, [P, ctypes.POINTER(ServeConfig)]),
    "stab_serve_submit": (I32, [P, U64, U32, U64, U64, P, U64, PU64]),
    "stab_serve_poll": (I32, [P, ctypes.POINTER(RequestStatus), SZ, ctypes.POINTER(SZ)]),
    "stab_serve_drain": (I32, [P, ctypes.c_double]),
    "stab_serve_stop": (I32, [P]),
    "stab_profile": (I32, [P, U32]),
    "stab_profile_read": (I32, [P, U32, ctypes.POINTER(KernelStats), I32]),
    "stab_launch_count": (I32, [P, PU64, I32]),
    "stab_engine_counters": (I32, [P, PU64, SZ, I32]),
    "stab_probe_copy": (I32, [P, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]),
}
EXPORTED = tuple(_SIGS)


def lib():
    """Load libstab.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2507_03092_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise StabError(rc, lib().stab_last_error().decode(errors="replace"))


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    raise TypeError("expected a torch tensor")


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def make_streams(mode=STREAM_BUFFER, coins=None, noise=None, seed=0, shot_offset=0):
    s = Streams()
    s.mode = mode
    s.seed = seed
    s.shot_offset = shot_offset
    if coins is not None:
        s.coins = coins.data_ptr()
        s.coin_words = coins.shape[-1]
    if noise is not None:
        s.noise = noise.data_ptr()
        s.noise_words = noise.shape[-1]
    return s


# ---------------------------------------------------------------- thin wrappers
def stab_create(device=0, stream=None):
    h = ctypes.c_void_p()
    _check(lib().stab_create(ctypes.byref(h), int(device), stream))
    return h


def stab_destroy(ctx):
    lib().stab_destroy(ctx)


def stab_set_stream(ctx, stream):
    _check(lib().stab_set_stream(ctx, stream))


def stab_sync(ctx):
    _check(lib().stab_sync(ctx))


def stab_compile(ctx, circ: C.Circuit) -> int:
    ops = np.ascontiguousarray(circ.ops, dtype=C.OP_DTYPE)
    params = np.ascontiguousarray(circ.params, dtype=np.float64).reshape(-1, 3)
    cid = ctypes.c_uint64()
    _check(lib().stab_compile(ctx, int(circ.n), _np_ptr(ops), len(ops), _np_ptr(params),
                              len(params), ctypes.byref(cid)))
    return int(cid.value)


def stab_circuit_info_get(ctx, cid) -> dict:
    info = CircuitInfo()
    _check(lib().stab_circuit_info_get(ctx, cid, ctypes.byref(info)))
    return info.as_dict()


def stab_compile_info(circ: C.Circuit) -> dict:
    """Validate and compile on the host only (no context, no GPU); returns
    the circuit info stab_compile would report."""
    ops = np.ascontiguousarray(circ.ops, dtype=C.OP_DTYPE)
    params = np.ascontiguousarray(circ.params, dtype=np.float64).reshape(-1, 3)
    info = CircuitInfo()
    _check(lib().stab_compile_info(int(circ.n), _np_ptr(ops), len(ops), _np_ptr(params), len(params),
                                   ctypes.byref(info)))
    return info.as_dict()


def stab_release_circuit(ctx, cid):
    _check(lib().stab_release_circuit(ctx, cid))


def stab_tableau_init(ctx, n, count=1):
    _check(lib().stab_tableau_init(ctx, int(n), int(count)))


def stab_apply_circuit(ctx, cid, streams: Streams, d_record):
    _check(lib().stab_apply_circuit(ctx, cid, ctypes.byref(streams), _ptr(d_record),
                                    d_record.shape[-1]))


def stab_get_tableau(ctx, index, n):
    W = (n + 63) // 64
    x = np.zeros((2 * n, W), np.uint64)
    z = np.zeros((2 * n, W), np.uint64)
    r = np.zeros(2 * n, np.uint8)
    _check(lib().stab_get_tableau(ctx, int(index), _np_ptr(x), _np_ptr(z), _np_ptr(r)))
    return x, z, r


def stab_set_tableau(ctx, index, x, z, r):
    x = np.ascontiguousarray(x, np.uint64)
    z = np.ascontiguousarray(z, np.uint64)
    r = np.ascontiguousarray(r, np.uint8)
    _check(lib().stab_set_tableau(ctx, int(index), _np_ptr(x), _np_ptr(z), _np_ptr(r)))


def stab_commute(ctx, index, d_px, d_pz, m, d_out):
    """Device tensors: d_px, d_pz uint64/int64 [m, ceil(n/64)]; d_out [m, 2 ceil(n/64)]."""
    _check(lib().stab_commute(ctx, int(index), _ptr(d_px), _ptr(d_pz), int(m), _ptr(d_out)))


def stab_sample(ctx, cid, shots, streams: Streams, d_record, engine=ENGINE_AUTO):
    _check(lib().stab_sample(ctx, cid, int(shots), ctypes.byref(streams), _ptr(d_record),
                             d_record.shape[-1], int(engine)))


def stab_sample_host(ctx, cid, shots, coins, noise, record_words, engine=ENGINE_AUTO):
    """Host numpy buffers in, host record out (copies happen inside the call)."""
    coins = np.ascontiguousarray(coins, np.uint64).reshape(shots, -1)
    noise = None if noise is None else np.ascontiguousarray(noise, np.uint32).reshape(shots, -1)
    rec = np.zeros((shots, record_words), np.uint64)
    _check(lib().stab_sample_host(ctx, cid, int(shots), _np_ptr(coins), coins.shape[1],
                                  _np_ptr(noise), 0 if noise is None else noise.shape[1],
                                  _np_ptr(rec), record_words, int(engine)))
    return rec


def stab_sample_batch(ctx, groups):
    arr = (JobGroup * len(groups))(*groups)
    _check(lib().stab_sample_batch(ctx, arr, len(groups)))


def stab_sample_batch_noalloc(ctx, groups):
    """stab_sample_batch without device allocation (fixed in-library scratch)."""
    arr = (JobGroup * len(groups))(*groups)
    _check(lib().stab_sample_batch_noalloc(ctx, arr, len(groups)))


def stab_autotune(ctx, cids, shots):
    arr = (ctypes.c_uint64 * len(cids))(*cids)
    _check(lib().stab_autotune(ctx, arr, len(cids), int(shots)))


def stab_get_tune(ctx, n) -> dict:
    t = Tune()
    _check(lib().stab_get_tune(ctx, int(n), ctypes.byref(t)))
    return t.as_dict()


def stab_set_tune(ctx, n, group_threads, tableaux_per_cta, words_per_thread):
    t = Tune(group_threads, tableaux_per_cta, words_per_thread, 0)
    _check(lib().stab_set_tune(ctx, int(n), ctypes.byref(t)))


def stab_serve_start(ctx, hbm_budget_bytes, max_inflight=64, n_streams=8, max_batch_requests=16):
    cfg = ServeConfig(int(hbm_budget_bytes), int(max_inflight), int(n_streams),
                      int(max_batch_requests), 0)
    _check(lib().stab_serve_start(ctx, ctypes.byref(cfg)))


def stab_serve_submit(ctx, cid, shots, seed, shot_offset, d_record) -> int:
    rid = ctypes.c_uint64()
    _check(lib().stab_serve_submit(ctx, cid, int(shots), int(seed), int(shot_offset),
                                   _ptr(d_record), d_record.shape[-1], ctypes.byref(rid)))
    return int(rid.value)


def stab_serve_poll(ctx, cap=4096):
    buf = (RequestStatus * cap)()
    nd = ctypes.c_size_t()
    _check(lib().stab_serve_poll(ctx, buf, cap, ctypes.byref(nd)))
    return [dict(req_id=int(b.req_id), status=int(b.status), shots=int(b.shots),
                 t_submit=b.t_submit, t_admit=b.t_admit, t_done=b.t_done)
            for b in buf[:nd.value]]


def stab_serve_drain(ctx, timeout_s=600.0):
    _check(lib().stab_serve_drain(ctx, float(timeout_s)))


def stab_serve_stop(ctx):
    _check(lib().stab_serve_stop(ctx))


def stab_profile(ctx, kind_mask):
    _check(lib().stab_profile(ctx, int(kind_mask)))


def stab_profile_read(ctx, kind, reset=True) -> dict:
    st = KernelStats()
    _check(lib().stab_profile_read(ctx, int(kind), ctypes.byref(st), 1 if reset else 0))
    return st.as_dict()


def stab_launch_count(ctx, reset=True) -> int:
    c = ctypes.c_uint64()
    _check(lib().stab_launch_count(ctx, ctypes.byref(c), 1 if reset else 0))
    return int(c.value)


COUNTER_NAMES = ("waves", "wave_ops", "det_in_wave_kernel", "det", "sum_K", "sum_A",
                 "pivot_recomputes", "rowsum_passes",
                 "cyc_pending", "cyc_cached", "cyc_col_rescans", "cyc_xs_rescans", "cyc_select",
                 "cyc_lists", "cyc_apply_single", "cyc_apply_multi", "w0_list_scan", "w0_list_pairs",
                 "w0_multi_walk", "xsupport_recomputes", "w0_multi_sort", "w0_multi_rows", "serial_waves", "dense_waves")


def stab_engine_counters(ctx, reset=True) -> dict:
    arr = (ctypes.c_uint64 * 24)()
    _check(lib().stab_engine_counters(ctx, arr, 24, 1 if reset else 0))
    return {k: int(v) for k, v in zip(COUNTER_NAMES, arr)}


def stab_probe_copy(ctx, nbytes, passes) -> float:
    """Read + write copy bandwidth (GB/s) over two buffers of nbytes/2 each."""
    out = ctypes.c_double(0.0)
    _check(lib().stab_probe_copy(ctx, int(nbytes), int(passes), ctypes.byref(out)))
    return float(out.value)


# ---------------------------------------------------------------- convenience
class Simulator:
    """A context on one device, bound to torch's current CUDA stream."""

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = stab_create(device, ctypes.c_void_p(stream))
        self._cids = {}

    def close(self):
        if self.ctx is not None:
            stab_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compile(self, circ: C.Circuit) -> int:
        return stab_compile(self.ctx, circ)

    def release(self, cid):
        stab_release_circuit(self.ctx, cid)

    def info(self, cid) -> dict:
        return stab_circuit_info_get(self.ctx, cid)

    def to_dev(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a).view(
            np.int64 if a.dtype == np.uint64 else np.int32)).to(self.device)

    def record_buffer(self, shots, words):
        return self.torch.zeros((shots, words), dtype=self.torch.int64, device=self.device)

    def sample(self, cid, circ, shots, coins=None, noise=None, seed=None, shot_offset=0,
               engine=ENGINE_AUTO, out=None):
        """Run `shots` shots; returns the device record tensor (int64 view of uint64)."""
        rec = out if out is not None else self.record_buffer(shots, circ.record_words)
        if seed is not None:
            st = make_streams(STREAM_SEEDED, seed=seed, shot_offset=shot_offset)
            stab_sample(self.ctx, cid, shots, st, rec, engine)
        else:
            dc = coins if coins is None or hasattr(coins, "data_ptr") else self.to_dev(coins)
            dn = noise if noise is None or hasattr(noise, "data_ptr") else self.to_dev(noise)
            st = make_streams(STREAM_BUFFER, coins=dc, noise=dn)
            stab_sample(self.ctx, cid, shots, st, rec, engine)
        return rec

    def sync(self):
        stab_sync(self.ctx)


def records_to_numpy(rec_tensor) -> np.ndarray:
    return rec_tensor.cpu().numpy().view(np.uint64)
