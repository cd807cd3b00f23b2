"""ctypes binding of libpanache.so: argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module only
converts Python arguments to the C ABI of ``include/panache.h``.  It raises
``ImportError`` when the compiled library is missing -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpanache.so")

OK, EINVAL, ENOMEM, EBUDGET, ECUDA, ETRUNC, ESTATE, EPOOL, ENODEV, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
EBUSY = -10
F32, F64, DEVICE = 1, 2, 0x100
PLAIN_FP64, MIXED = 0, 1
TOPK_GLOBAL, TOPK_PER_LENGTH = 0, 1
FLAG_EXHAUSTIVE_SIEVE, FLAG_NO_SIEVE, FLAG_NO_COMPLETION, FLAG_TIMING, FLAG_INDEX_ONLY = 0x1, 0x2, 0x4, 0x8, 0x10
FLAG_FP64_ANCHORS = 0x20
FLAG_GRAPH = 0x40
FLAG_HALF_FEATURES = 0x80
FLAG_WARM_START = 0x100
FLAG_NO_REFINE = 0x200
FLAG_GRAM_SEARCH = 0x800
FLAG_TOPK_SIEVE = 0x1000
FLAG_NO_FOCUS_SIEVE = 0x2000
FLAG_SIEVE_GRAM = 0x400
NOALLOC_NEED_MAX = 6300   # largest k (m + 1) of panache_topk_row_noalloc
FAULT_NONE, FAULT_ALLOC, FAULT_COPY, FAULT_TC_WAIT = 0, 1, 2, 3

EXPORTED = ("panache_default_config", "panache_create", "panache_destroy", "panache_set_stream", "panache_pmp",
            "panache_pmp_batch", "panache_pmp_anchor_shard", "panache_pmp_from_rows", "panache_stream_open", "panache_append", "panache_stream_topk",
            "panache_stream_length", "panache_stream_close", "panache_stream_checkpoint", "panache_last_stats",
            "panache_profile_rows",
            "panache_anchor_state", "panache_query_levels", "panache_query_candidates", "panache_projections", "panache_calibrate_width",
            "panache_strerror",
            "panache_topk_row_noalloc", "panache_alu_peak", "panache_kernel_times", "panache_inject_fault",
            "panache_server_create", "panache_server_destroy", "panache_server_submit", "panache_server_wait",
            "panache_server_stream_open", "panache_server_append", "panache_server_stream_topk",
            "panache_server_stream_close", "panache_server_get_stats", "panache_server_set_deadline")


class Config(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_uint32), ("gamma", ctypes.c_uint32), ("stride", ctypes.c_uint32),
                ("K", ctypes.c_uint32), ("B", ctypes.c_uint32), ("d0", ctypes.c_uint32),
                ("probe_cap", ctypes.c_uint32), ("sieve_w", ctypes.c_uint32), ("dm", ctypes.c_uint32),
                ("dp", ctypes.c_uint32), ("rounds", ctypes.c_uint32), ("precision", ctypes.c_uint32),
                ("topk_mode", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("beta", ctypes.c_uint32), ("seed_mult", ctypes.c_uint32), ("grid_mult", ctypes.c_uint32),
                ("refine_mult", ctypes.c_uint32), ("_reserved", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("hbm_budget_bytes", ctypes.c_uint64),
                ("lambda_", ctypes.c_double), ("eps0", ctypes.c_double)]


class Motif(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("_pad", ctypes.c_int32), ("i", ctypes.c_int64), ("j", ctypes.c_int64),
                ("d", ctypes.c_double)]


MOTIF_DTYPE = np.dtype([("m", np.int32), ("_pad", np.int32), ("i", np.int64), ("j", np.int64), ("d", np.float64)])


class Request(ctypes.Structure):
    _fields_ = [("series", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("_pad", ctypes.c_int32),
                ("n", ctypes.c_int64), ("m_min", ctypes.c_int32), ("m_max", ctypes.c_int32),
                ("k", ctypes.c_int32), ("excl", ctypes.c_int32)]


STEP_NAMES = ("upload", "moments", "features", "directory", "search", "sieve", "completion", "select")
KERNEL_NAMES = ("anchor_tc", "features", "search", "sieve", "complete", "select", "refine", "topk_sieve")
KERNEL_TIMES = len(KERNEL_NAMES)


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "queries", "candidates", "exact_stream", "exact_sieve", "exact_completion", "hot_classes",
        "completion_rounds", "device_bytes", "kernel_launches", "waves", "refine_passes", "exact_refine")] + \
        [("step_ms", ctypes.c_double * 8)]


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "submitted", "completed", "failed", "queued", "batches", "windows_lengths", "budget_bytes",
        "peak_reserved_bytes")] + [("max_concurrent_batches", ctypes.c_uint32), ("_pad", ctypes.c_uint32)] + \
        [(name, ctypes.c_double) for name in ("span_ms", "p50_ms", "p99_ms", "mean_ms")] + \
        [("refused", ctypes.c_uint64), ("snap_p50_ms", ctypes.c_double), ("snap_p99_ms", ctypes.c_double),
         ("refused_snapshots", ctypes.c_uint64)]


_lib = None


def lib():
    """Loads the compiled library; raises ImportError when it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_17481_b300.build` "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32)
        L.panache_default_config.argtypes = [ctypes.POINTER(Config)]
        L.panache_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
        L.panache_destroy.argtypes = [vp]
        L.panache_destroy.restype = None
        L.panache_set_stream.argtypes = [vp, vp]
        L.panache_pmp.argtypes = [vp, vp, i32, i64, i32, i32, i32, i32, vp, i64, ctypes.POINTER(i64)]
        L.panache_pmp_batch.argtypes = [vp, vp, i32, vp, i64, vp]
        L.panache_pmp_anchor_shard.argtypes = [vp, vp, i32, i64, i32, i32, i32, i32, i32, i32, vp, i64]
        L.panache_pmp_from_rows.argtypes = [vp, vp, i32, i64, i32, i32, i32, i32, vp, vp, i64, ctypes.POINTER(i64)]
        L.panache_stream_open.argtypes = [vp, i32, i32, i32, i32, ctypes.POINTER(vp)]
        L.panache_append.argtypes = [vp, vp, i32, i64]
        L.panache_stream_topk.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
        L.panache_stream_length.argtypes = [vp]
        L.panache_stream_length.restype = i64
        L.panache_stream_close.argtypes = [vp]
        L.panache_stream_checkpoint.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
        L.panache_stream_close.restype = None
        L.panache_last_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.panache_profile_rows.argtypes = [vp, i32, vp, i64]
        L.panache_anchor_state.argtypes = [vp, i32, i32, ctypes.POINTER(i32), vp, vp, i64]
        L.panache_query_levels.argtypes = [vp, i32, i32, vp, vp, i64]
        L.panache_query_candidates.argtypes = [vp, i32, i32, vp, i32, vp, i32, vp]
        L.panache_kernel_times.argtypes = [vp, vp, vp, i32]
        L.panache_alu_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        L.panache_inject_fault.argtypes = [i32, i32]
        L.panache_projections.argtypes = [ctypes.POINTER(Config), i32, vp, i64]
        L.panache_topk_row_noalloc.argtypes = [vp, i64, i32, vp, i32, ctypes.c_double, vp, vp, vp]
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.panache_server_create.argtypes = [ctypes.POINTER(Config), i32, ctypes.c_uint64, ctypes.POINTER(vp)]
        L.panache_server_destroy.argtypes = [vp]
        L.panache_server_destroy.restype = None
        L.panache_server_submit.argtypes = [vp, vp, i32, i64, i32, i32, i32, i32, u64p]
        L.panache_server_wait.argtypes = [vp, ctypes.c_uint64, i32, vp, i64, ctypes.POINTER(i64),
                                          ctypes.POINTER(ctypes.c_double)]
        L.panache_server_stream_open.argtypes = [vp, i32, i32, i32, i32, u64p]
        L.panache_server_append.argtypes = [vp, ctypes.c_uint64, vp, i32, i64]
        L.panache_server_stream_topk.argtypes = [vp, ctypes.c_uint64, u64p]
        L.panache_server_stream_close.argtypes = [vp, ctypes.c_uint64]
        L.panache_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.panache_server_set_deadline.argtypes = [vp, ctypes.c_double]
        L.panache_calibrate_width.argtypes = [vp, vp, i32, i64, i32, i32, ctypes.c_double, ctypes.POINTER(i32),
                                              vp, vp]
        L.panache_strerror.argtypes = [ctypes.c_int]
        L.panache_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


class PanacheError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {lib().panache_strerror(code).decode()} ({code})")


def _check(rc: int, what: str):
    if rc != OK:
        raise PanacheError(rc, what)


def default_config(**over) -> Config:
    c = Config()
    _check(lib().panache_default_config(ctypes.byref(c)), "default_config")
    for k, v in over.items():
        setattr(c, "lambda_" if k == "lam" else k, v)
    return c


def _series_arg(x):
    """(pointer, dtype flag, n, keepalive) for a numpy array or a CUDA tensor."""
    if hasattr(x, "is_cuda") and x.is_cuda:
        import torch
        if x.dtype not in (torch.float32, torch.float64) or not x.is_contiguous():
            raise ValueError("series tensor must be contiguous float32/float64")
        return ctypes.c_void_p(x.data_ptr()), (F32 if x.dtype == torch.float32 else F64) | DEVICE, x.numel(), x
    a = np.asarray(x)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    a = np.ascontiguousarray(a)
    return a.ctypes.data_as(ctypes.c_void_p), F32 if a.dtype == np.float32 else F64, a.shape[0], a


def projections(a: int, config: Config | None = None) -> np.ndarray:
    """The FP32 projections [B+1][32] a context with `config` draws for anchor length a."""
    cfg = config if config is not None else default_config()
    g = np.empty((cfg.B + 1, 32), dtype=np.float32)
    _check(lib().panache_projections(ctypes.byref(cfg), a, g.ctypes.data_as(ctypes.c_void_p), g.size),
           "projections")
    return g


class Context:
    """One engine context on the current CUDA device."""

    def __init__(self, config: Config | None = None, **over):
        cfg = config if config is not None else default_config(**over)
        self._h = ctypes.c_void_p()
        _check(lib().panache_create(ctypes.byref(cfg), ctypes.byref(self._h)), "create")
        self.config = cfg

    def close(self):
        if self._h:
            lib().panache_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr: int | None):
        _check(lib().panache_set_stream(self._h, ctypes.c_void_p(stream_ptr or 0)), "set_stream")

    def pmp(self, x, m_min: int, m_max: int, k: int, excl: int, out_cap: int | None = None) -> np.ndarray:
        ptr, dt, n, keep = _series_arg(x)
        L = max(0, m_max - m_min + 1)
        cap = out_cap if out_cap is not None else max(0, k) * L
        out = np.zeros(max(cap, 1), dtype=MOTIF_DTYPE)
        ln = ctypes.c_int64()
        rc = lib().panache_pmp(self._h, ptr, dt, n, m_min, m_max, k, excl,
                               out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(ln))
        _check(rc, "pmp")
        del keep
        return out[:ln.value]

    def pmp_anchor_shard(self, x, m_min: int, m_max: int, k: int, excl: int, rank: int, world: int) -> np.ndarray:
        """This rank's profile rows [L][n] (packed keys) after its anchors' search and sieve."""
        ptr, dt, n, keep = _series_arg(x)
        L = m_max - m_min + 1
        rows = np.empty((L, n), dtype=np.uint64)
        _check(lib().panache_pmp_anchor_shard(self._h, ptr, dt, n, m_min, m_max, k, excl, rank, world,
                                              rows.ctypes.data_as(ctypes.c_void_p), rows.size), "pmp_anchor_shard")
        del keep
        return rows

    def pmp_from_rows(self, x, m_min: int, m_max: int, k: int, excl: int, rows: np.ndarray) -> np.ndarray:
        """Motifs from merged profile rows [L][n]: completion, refinement and selection."""
        ptr, dt, n, keep = _series_arg(x)
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        L = m_max - m_min + 1
        if rows.shape != (L, n):
            raise ValueError(f"rows must have shape {(L, n)}")
        cap = max(0, k) * L
        out = np.zeros(max(cap, 1), dtype=MOTIF_DTYPE)
        ln = ctypes.c_int64()
        _check(lib().panache_pmp_from_rows(self._h, ptr, dt, n, m_min, m_max, k, excl,
                                           rows.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                           cap, ctypes.byref(ln)), "pmp_from_rows")
        del keep
        return out[:ln.value]

    def pmp_batch(self, series: list, params: list[tuple[int, int, int, int]], out_cap_per_req: int | None = None):
        reqs = (Request * len(series))()
        keep = []
        cap = out_cap_per_req or max(1, max(k * (mx - mn + 1) for (mn, mx, k, _) in params))
        for r, (x, (mn, mx, k, ex)) in enumerate(zip(series, params)):
            ptr, dt, n, kp = _series_arg(x)
            keep.append(kp)
            reqs[r].series, reqs[r].dtype, reqs[r].n = ptr, dt, n
            reqs[r].m_min, reqs[r].m_max, reqs[r].k, reqs[r].excl = mn, mx, k, ex
        out = np.zeros(cap * len(series), dtype=MOTIF_DTYPE)
        lens = np.zeros(len(series), dtype=np.int64)
        rc = lib().panache_pmp_batch(self._h, ctypes.cast(reqs, ctypes.c_void_p), len(series),
                                     out.ctypes.data_as(ctypes.c_void_p), cap,
                                     lens.ctypes.data_as(ctypes.c_void_p))
        _check(rc, "pmp_batch")
        return [out[r * cap: r * cap + lens[r]] for r in range(len(series))]

    def stats(self) -> dict:
        s = Stats()
        _check(lib().panache_last_stats(self._h, ctypes.byref(s)), "last_stats")
        out = {name: int(getattr(s, name)) for name, _ in Stats._fields_ if name != "step_ms"}
        out["step_ms"] = {nm: float(s.step_ms[t]) for t, nm in enumerate(STEP_NAMES)}
        return out

    def kernel_times(self) -> dict:
        """{kernel: (ms, launches)} of the last request made with FLAG_TIMING."""
        ms = np.zeros(KERNEL_TIMES)
        ln = np.zeros(KERNEL_TIMES, dtype=np.uint64)
        _check(lib().panache_kernel_times(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                          ln.ctypes.data_as(ctypes.c_void_p), KERNEL_TIMES), "kernel_times")
        return {nm: (float(ms[k]), int(ln[k])) for k, nm in enumerate(KERNEL_NAMES)}

    def profile_rows(self, series_index: int, n: int, L: int) -> np.ndarray:
        keys = np.empty(n * L, dtype=np.uint64)
        _check(lib().panache_profile_rows(self._h, series_index, keys.ctypes.data_as(ctypes.c_void_p), keys.size),
               "profile_rows")
        return keys.reshape(L, n)

    def anchor_state(self, series_index: int, anchor_index: int, nw: int):
        a = ctypes.c_int32()
        F = np.empty((nw, 32), dtype=np.float32)
        sig = np.empty(nw, dtype=np.uint32)
        _check(lib().panache_anchor_state(self._h, series_index, anchor_index, ctypes.byref(a),
                                          F.ctypes.data_as(ctypes.c_void_p), sig.ctypes.data_as(ctypes.c_void_p),
                                          nw), "anchor_state")
        return a.value, F, sig

    def query_levels(self, series_index: int, anchor_index: int, nw: int):
        """(population, depth) per window of one anchor of the last request, -1 where not searched."""
        pop = np.empty(max(1, nw), dtype=np.int32)
        dep = np.empty(max(1, nw), dtype=np.int32)
        _check(lib().panache_query_levels(self._h, series_index, anchor_index, pop.ctypes.data_as(ctypes.c_void_p),
                                          dep.ctypes.data_as(ctypes.c_void_p), nw), "query_levels")
        return pop[:nw], dep[:nw]

    def query_candidates(self, series_index: int, anchor_index: int, qs, cap: int = 512):
        """Candidate lists of the listed queries of one anchor of the last request: list of arrays (None if skipped)."""
        qs = np.ascontiguousarray(qs, dtype=np.int64)
        cand = np.zeros((max(1, len(qs)), cap), dtype=np.uint32)
        cnt = np.zeros(max(1, len(qs)), dtype=np.int32)
        _check(lib().panache_query_candidates(self._h, series_index, anchor_index, qs.ctypes.data_as(ctypes.c_void_p),
                                              len(qs), cand.ctypes.data_as(ctypes.c_void_p), cap,
                                              cnt.ctypes.data_as(ctypes.c_void_p)), "query_candidates")
        return [None if cnt[i] < 0 else cand[i, :min(cap, cnt[i])].copy() for i in range(len(qs))]

    def projections(self, a: int) -> np.ndarray:
        return projections(a, self.config)

    def calibrate_width(self, x, m_min: int, m_max: int, eta: float = 0.0):
        """(K, energy[K=2..16], collision_prob[K=2..16]): the spectral-width calibration of series x."""
        ptr, dt, n, keep = _series_arg(x)
        K = ctypes.c_int32()
        e = np.zeros(15)
        c = np.zeros(15)
        _check(lib().panache_calibrate_width(self._h, ptr, dt, n, m_min, m_max, eta, ctypes.byref(K),
                                             e.ctypes.data_as(ctypes.c_void_p), c.ctypes.data_as(ctypes.c_void_p)),
               "calibrate_width")
        del keep
        return K.value, e, c

    def stream(self, m_min: int, m_max: int, k: int, excl: int) -> "Stream":
        return Stream(self, m_min, m_max, k, excl)


class Stream:
    """A live series with its index resident on the device: appends of any size, top-k on request."""

    def __init__(self, ctx: Context, m_min: int, m_max: int, k: int, excl: int):
        self.ctx = ctx
        self.L, self.k = m_max - m_min + 1, k
        self._h = ctypes.c_void_p()
        _check(lib().panache_stream_open(ctx._h, m_min, m_max, k, excl, ctypes.byref(self._h)), "stream_open")

    def append(self, chunk):
        ptr, dt, n, keep = _series_arg(chunk)
        _check(lib().panache_append(self._h, ptr, dt, n), "append")
        del keep

    def __len__(self):
        return int(lib().panache_stream_length(self._h))

    def checkpoint(self) -> np.ndarray:
        """The stream's samples (FP64): appending them to a fresh stream resumes it."""
        n = len(self)
        out = np.zeros(max(1, n), dtype=np.float64)
        ln = ctypes.c_int64()
        _check(lib().panache_stream_checkpoint(self._h, out.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(ln)),
               "stream_checkpoint")
        return out[:ln.value]

    def topk(self) -> np.ndarray:
        cap = self.k * self.L
        out = np.zeros(cap, dtype=MOTIF_DTYPE)
        ln = ctypes.c_int64()
        _check(lib().panache_stream_topk(self._h, out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(ln)),
               "stream_topk")
        return out[:ln.value]

    def close(self):
        if self._h:
            lib().panache_stream_close(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server: continuous batching over `slots` concurrent streams under an HBM budget."""

    def __init__(self, slots: int = 4, hbm_budget_bytes: int = 0, config: Config | None = None, **over):
        cfg = config if config is not None else default_config(**over)
        self._h = ctypes.c_void_p()
        _check(lib().panache_server_create(ctypes.byref(cfg), slots, hbm_budget_bytes, ctypes.byref(self._h)),
               "server_create")
        self.config = cfg
        self._caps: dict[int, int] = {}

    def submit(self, x, m_min: int, m_max: int, k: int, excl: int) -> int:
        a = np.ascontiguousarray(np.asarray(x))
        if a.dtype not in (np.float32, np.float64):
            a = a.astype(np.float64)
        t = ctypes.c_uint64()
        _check(lib().panache_server_submit(self._h, a.ctypes.data_as(ctypes.c_void_p), F32 if a.dtype == np.float32
                                           else F64, a.shape[0], m_min, m_max, k, excl, ctypes.byref(t)), "submit")
        self._caps[t.value] = k * (m_max - m_min + 1)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(motifs, latency_ms); raises PanacheError (ETIMEOUT when not ready in time)."""
        cap = max(1, self._caps.get(ticket, 4096))
        out = np.zeros(cap, dtype=MOTIF_DTYPE)
        ln = ctypes.c_int64()
        lat = ctypes.c_double()
        _check(lib().panache_server_wait(self._h, ticket, timeout_ms, out.ctypes.data_as(ctypes.c_void_p), cap,
                                         ctypes.byref(ln), ctypes.byref(lat)), "wait")
        self._caps.pop(ticket, None)
        return out[:ln.value], lat.value

    def stream_open(self, m_min: int, m_max: int, k: int, excl: int) -> int:
        sid = ctypes.c_uint64()
        _check(lib().panache_server_stream_open(self._h, m_min, m_max, k, excl, ctypes.byref(sid)), "stream_open")
        self._caps[("s", sid.value)] = k * (m_max - m_min + 1)
        return sid.value

    def append(self, sid: int, chunk):
        a = np.ascontiguousarray(np.asarray(chunk))
        if a.dtype not in (np.float32, np.float64):
            a = a.astype(np.float64)
        _check(lib().panache_server_append(self._h, sid, a.ctypes.data_as(ctypes.c_void_p),
                                           F32 if a.dtype == np.float32 else F64, a.shape[0]), "append")

    def stream_topk(self, sid: int) -> int:
        t = ctypes.c_uint64()
        _check(lib().panache_server_stream_topk(self._h, sid, ctypes.byref(t)), "stream_topk")
        self._caps[t.value] = self._caps.get(("s", sid), 4096)
        return t.value

    def stream_close(self, sid: int):
        _check(lib().panache_server_stream_close(self._h, sid), "stream_close")
        self._caps.pop(("s", sid), None)

    def set_deadline(self, deadline_ms: float):
        """Deadline admission: submissions predicted to wait longer are refused (EBUSY); 0 turns it off."""
        _check(lib().panache_server_set_deadline(self._h, deadline_ms), "set_deadline")

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().panache_server_get_stats(self._h, ctypes.byref(s)), "server_stats")
        return {name: getattr(s, name) for name, _ in ServerStats._fields_ if name != "_pad"}

    def close(self):
        if self._h:
            lib().panache_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MOTIF_BYTES = ctypes.sizeof(Motif)


def topk_row_noalloc(x_dev, keys_dev, m: int, k: int, eps0: float, out_dev, count_dev, stream_ptr: int = 0):
    """Selection of one length row with no device allocation (all buffers are the caller's device tensors).

    x_dev: contiguous float64 samples; keys_dev: contiguous int64/uint64 packed keys, one per sample;
    out_dev: contiguous device buffer of at least k motifs (32 bytes each); count_dev: contiguous int32
    device tensor.  All four must sit on the current CUDA device.  Anything else raises ValueError before
    the library is called, since the kernels would read or write past the caller's buffers.  Returns the
    library's status code."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("x", x_dev), ("keys", keys_dev), ("out", out_dev), ("count", count_dev)):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if x_dev.dtype != torch.float64:
        raise ValueError("x must be float64")
    if keys_dev.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise ValueError("keys must be int64 or uint64")
    if keys_dev.numel() != x_dev.numel():
        raise ValueError("keys must hold one key per sample of x")
    if k < 1 or out_dev.numel() * out_dev.element_size() < k * MOTIF_BYTES:
        raise ValueError(f"out must hold at least k = {k} motifs of {MOTIF_BYTES} bytes")
    if count_dev.dtype != torch.int32 or count_dev.numel() < 1:
        raise ValueError("count must be an int32 tensor of at least one element")
    return lib().panache_topk_row_noalloc(ctypes.c_void_p(x_dev.data_ptr()), x_dev.numel(), m,
                                          ctypes.c_void_p(keys_dev.data_ptr()), k, eps0,
                                          ctypes.c_void_p(out_dev.data_ptr()), ctypes.c_void_p(count_dev.data_ptr()),
                                          ctypes.c_void_p(stream_ptr))


def inject_fault(kind: int, after: int = 0):
    """Arms one host-made failure of a later operation (test hook; FAULT_NONE disarms)."""
    _check(lib().panache_inject_fault(kind, after), "inject_fault")


def alu_peak(kind: int) -> float:
    """Measured TFLOP/s of one pipe on the current device: 0 FP32 FMA, 1 packed FP32 FMA, 2 FP64 FMA."""
    t = ctypes.c_double()
    _check(lib().panache_alu_peak(kind, ctypes.byref(t)), "alu_peak")
    return t.value


def unpack_keys(keys: np.ndarray):
    """(distance, neighbour) arrays from packed profile keys; empty cells give (inf, -1)."""
    keys = np.asarray(keys, dtype=np.uint64)
    empty = keys == np.uint64(0xFFFFFFFFFFFFFFFF)
    mask = np.uint64((1 << 26) - 1)
    d = (keys & ~mask).view(np.float64).copy()
    j = (keys & mask).astype(np.int64)
    d[empty] = np.inf
    j[empty] = -1
    return d, j
