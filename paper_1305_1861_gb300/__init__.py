"""GB300-native frequent k-mer counting (Turtle, arXiv:1305.1861).

The compute path lives in ``libturtle.so`` (hand-written sm_103a CUDA kernels
behind the C ABI declared in ``include/turtle.h``).  This package is a thin
ctypes binding with the same names: it marshals arguments (NumPy arrays, torch
CUDA tensors and streams to plain pointers) and raises on error codes.  Every
step of the path runs in the library's kernels; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "TurtleError", "Params", "Context", "Server", "load", "build", "turtle_count", "turtle_count_batch",
    "turtle_strerror", "turtle_trim", "STAGES",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libturtle.so")
_lib = None

u64 = ctypes.c_uint64
u32 = ctypes.c_uint32
_p = ctypes.c_void_p

TURTLE_OK = 0
ERRORS = {-1: "TURTLE_E_ARG", -2: "TURTLE_E_NOMEM", -3: "TURTLE_E_CUDA", -4: "TURTLE_E_OVERFLOW",
          -5: "TURTLE_E_TIMEOUT", -6: "TURTLE_E_BUSY", -7: "TURTLE_E_DEVICE", -8: "TURTLE_E_NODEV",
          -9: "TURTLE_E_CAPACITY", -10: "TURTLE_E_TOO_LARGE"}
STAGES = ["pack", "valid", "filter", "hist", "sort", "rle", "table", "recount", "threshold", "merge"]
HOST_PHASES = ["input", "path", "touch", "output"]


class TurtleError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s failed: %s (%s)" % (where, ERRORS.get(code, code), turtle_strerror(code)))


class Params(ctypes.Structure):
    _fields_ = [("struct_size", u32), ("filter_bits_per_window", ctypes.c_float), ("pattern_bits", u32),
                ("n_patterns", u32), ("pattern_seed", u64), ("timing", u32), ("l2_fetch_bytes", u32),
                ("recount_windows", u32), ("member_filter", u32), ("budget_mib", u32),
                ("stream_chunk_mib", u32), ("sort_tile", u32),
                ("compact", u32), ("bucket_slots", u32),
                ("cturtle_bits_per_window", u32), ("hash_slots_log2", u32), ("shard_count", u32),
                ("shard_index", u32), ("probe_order", u32), ("bucket_windows", u32), ("autotune", u32),
                ("host_transfer", u32), ("batch_mixed", u32)]

    @classmethod
    def default(cls, **kw) -> "Params":
        p = cls()
        load().turtle_params_default(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p


class TuneReport(ctypes.Structure):
    _fields_ = [("evaluations", u32), ("cached", u32), ("default_ms", ctypes.c_float), ("best_ms", ctypes.c_float),
                ("sample_bases", u64)]


TUNE_TIMER = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p)


class _Reads(ctypes.Structure):
    _fields_ = [("bases", _p), ("offsets", _p), ("n_reads", u64)]


class _Result(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n", u64), ("keys", ctypes.POINTER(u64)), ("counts", ctypes.POINTER(u32)),
                ("n_windows", u64)]


class _DeviceResult(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("key_words", ctypes.c_int), ("n", u64), ("keys", _p), ("counts", _p),
                ("n_windows", u64)]


class Stats(ctypes.Structure):
    _fields_ = [("n_windows", u64), ("n_candidates", u64), ("n_firsts", u64), ("n_unique", u64), ("n_out", u64),
                ("filter_bytes", u64), ("table_bytes", u64), ("scratch_bytes", u64), ("sort_passes", u32),
                ("super_partitions", u32), ("launches", u32), ("stage_launches", u32 * 10), ("stage_ms", ctypes.c_float * 10),
                ("host_ms", ctypes.c_float * 4), ("h2d_ms", ctypes.c_float), ("h2d_bytes", u64), ("d2h_bytes", u64),
                ("chunks", u32), ("host_locked", u32), ("transfer_gbs", ctypes.c_float * 3), ("pad_", u32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in ("stage_launches", "stage_ms", "host_ms", "pad_", "transfer_gbs")}
        d["transfer_gbs"] = {n: round(float(self.transfer_gbs[i]), 1)
                             for i, n in enumerate(("pageable", "page_locking", "page_locked_copy"))}
        d["stage_launches"] = {STAGES[i]: int(self.stage_launches[i]) for i in range(len(STAGES))}
        d["stage_ms"] = {STAGES[i]: float(self.stage_ms[i]) for i in range(len(STAGES))}
        d["host_ms"] = {HOST_PHASES[i]: float(self.host_ms[i]) for i in range(4)}
        return d


def build(force: bool = False) -> str:
    from . import _nvcc
    return _nvcc.build(force=force)


def load():
    """Load libturtle.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libturtle.so not built: run paper_1305_1861_gb300.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(_LIB_PATH)
    sig = {
        "turtle_params_default": (None, [_p]),
        "turtle_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "turtle_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
        "turtle_count": (ctypes.c_int, [_p, ctypes.c_int, u32, _p]),
        "turtle_count_ex": (ctypes.c_int, [_p, ctypes.c_int, u32, _p, _p, _p]),
        "turtle_result_free": (None, [_p]),
        "turtle_ctx_create": (ctypes.c_int, [ctypes.c_int, _p]),
        "turtle_ctx_destroy": (None, [_p]),
        "turtle_ctx_stats": (ctypes.c_int, [_p, _p]),
        "turtle_shard_bounds": (ctypes.c_int, [_p, u32, u32, _p]),
        "turtle_ctx_pool_bytes": (ctypes.c_int, [_p, _p, _p]),
        "turtle_ctx_trim": (None, [_p]),
        "turtle_test_inject": (ctypes.c_int, [ctypes.c_int, u64]),
        "turtle_tune_select": (ctypes.c_int, [_p, _p, _p, _p, _p]),
        "turtle_autotune": (ctypes.c_int, [_p, _p, u64, _p, u64, ctypes.c_int, u32, _p, _p, _p, _p]),
        "turtle_tune_cache_clear": (None, []),
        "turtle_trim": (None, []),
        "turtle_ctx_count": (ctypes.c_int, [_p, _p, ctypes.c_int, u32, _p, _p, _p]),
        "turtle_count_device": (ctypes.c_int, [_p, _p, u64, _p, u64, ctypes.c_int, u32, _p, _p, _p]),
        "turtle_frequent": (ctypes.c_int, [_p, ctypes.c_int, _p, _p, _p]),
        "turtle_frequent_device": (ctypes.c_int, [_p, _p, u64, _p, u64, ctypes.c_int, _p, _p, _p]),
        "turtle_extract": (ctypes.c_int, [_p, _p, u64, _p, u64, ctypes.c_int, _p, _p, _p, _p]),
        "turtle_filter": (ctypes.c_int, [_p, _p, u64, ctypes.c_int, _p, u64, _p, ctypes.c_int, _p, _p]),
        "turtle_sort_compact": (ctypes.c_int, [_p, _p, u64, ctypes.c_int, ctypes.c_int, _p, _p, _p, _p]),
        "turtle_sort_compact_noalloc": (ctypes.c_int, [_p, u64, ctypes.c_int, ctypes.c_int, _p, _p, _p, _p]),
        "turtle_count_batch": (ctypes.c_int, [_p, ctypes.c_size_t, _p, _p, _p]),
        "turtle_server_create": (ctypes.c_int, [ctypes.c_int, u64, ctypes.c_int, _p, _p]),
        "turtle_server_create_ex": (ctypes.c_int, [ctypes.c_int, u64, ctypes.c_int, ctypes.c_int, _p, _p]),
        "turtle_submit": (ctypes.c_int, [_p, _p, _p]),
        "turtle_poll": (ctypes.c_int, [_p, u64, ctypes.c_int, _p, _p]),
        "turtle_server_stats_get": (ctypes.c_int, [_p, _p]),
        "turtle_server_destroy": (None, [_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def turtle_trim():
    """Give back the device memory the library's internal contexts keep unused, and recycled host results."""
    load().turtle_trim()


def turtle_strerror(code: int) -> str:
    return load().turtle_strerror(code).decode()


def _check(rc: int, where: str):
    if rc != TURTLE_OK:
        raise TurtleError(rc, where)


def _np(a, dtype):
    a = np.ascontiguousarray(a)
    if a.dtype != dtype:
        a = a.astype(dtype)
    return a


def _shape_keys(flat: np.ndarray, n: int, k: int) -> np.ndarray:
    return flat.reshape(n, 2) if k > 32 else flat


class _ResultOwner:
    """Holds a library-allocated turtle_result; frees it when the last NumPy view goes away."""

    def __init__(self, lib, res):
        self._lib, self._res = lib, res

    def __del__(self):
        self._lib.turtle_result_free(ctypes.byref(self._res))


class _View:
    """Array interface over one buffer of a turtle_result; keeps its owner alive."""

    def __init__(self, owner, ptr, n, typestr):
        self._owner = owner
        self.__array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


def _take(lib, res, k):
    """(keys, counts, n_windows) viewing the library's buffers without a copy; the result is freed with them."""
    w = 2 if k > 32 else 1
    n = int(res.n)
    nw = int(res.n_windows)
    if n == 0:
        lib.turtle_result_free(ctypes.byref(res))
        return _shape_keys(np.zeros(0, dtype=np.uint64), 0, k), np.zeros(0, np.uint32), nw
    owner = _ResultOwner(lib, res)
    keys = np.asarray(_View(owner, ctypes.cast(res.keys, ctypes.c_void_p).value, n * w, "<u8"))
    cptr = ctypes.cast(res.counts, ctypes.c_void_p).value
    counts = np.asarray(_View(owner, cptr, n, "<u4")) if cptr else None
    return _shape_keys(keys, n, k), counts, nw


def turtle_count(bases, offsets, k: int, min_count: int = 2, params: Params | None = None, stream=None):
    """Host-memory form: (keys, counts, n_windows) as NumPy arrays, keys uint64[n] or uint64[n, 2] (hi, lo)."""
    lib = load()
    b = _np(bases, np.uint8)
    o = _np(offsets, np.uint64)
    reads = _Reads(b.ctypes.data if b.size else None, o.ctypes.data, o.size - 1)
    res = _Result()
    rc = lib.turtle_count_ex(ctypes.byref(reads), k, min_count, ctypes.byref(params) if params else None,
                             _stream_ptr(stream), ctypes.byref(res))
    _check(rc, "turtle_count")
    return _take(lib, res, k)


def turtle_frequent(bases, offsets, k: int, params: Params | None = None, stream=None):
    """cTurtle (Sec. 2.2): (keys, n_windows) of the k-mers seen at least twice, approximate, no counts;
    keys ascending, uint64[n] or uint64[n, 2] (hi, lo)."""
    lib = load()
    b = _np(bases, np.uint8)
    o = _np(offsets, np.uint64)
    reads = _Reads(b.ctypes.data if b.size else None, o.ctypes.data, o.size - 1)
    res = _Result()
    rc = lib.turtle_frequent(ctypes.byref(reads), k, ctypes.byref(params) if params else None, _stream_ptr(stream),
                             ctypes.byref(res))
    _check(rc, "turtle_frequent")
    keys, _, nw = _take(lib, res, k)
    return keys, nw


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def turtle_sort_compact_noalloc(keys, key_bits: int, unique, counts, stream=None) -> int:
    """Allocation-free sort-and-compact into caller-owned CUDA buffers; returns n_unique.

    For callers that must not allocate device memory: the library's scratch is a
    fixed array inside its device image (limits: TURTLE_NOALLOC_MAX_KEYS64 /
    TURTLE_NOALLOC_MAX_KEYS128 keys). Calls that overlap on the GPU race.
    """
    n = keys.shape[0]
    w = 2 if keys.dim() == 2 else 1
    nu = u64()
    rc = load().turtle_sort_compact_noalloc(keys.data_ptr(), n, w, key_bits, unique.data_ptr(), counts.data_ptr(),
                                            ctypes.byref(nu), _stream_ptr(stream))
    _check(rc, "turtle_sort_compact_noalloc")
    return int(nu.value)


class _Job(ctypes.Structure):
    _fields_ = [("bases", _p), ("offsets", _p), ("n_reads", u64), ("k", ctypes.c_int), ("min_count", u32)]


class JobTimes(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, u64) for n in ("budget_bytes", "admitted_bytes", "peak_admitted_bytes", "submitted", "completed",
                                   "failed", "queued", "running", "peak_running", "peak_queued", "batches",
                                   "largest_batch", "executors", "peak_running_batches")]


def turtle_count_batch(jobs, params: Params | None = None, stream=None):
    """Batched form. jobs: [(bases, offsets, k, min_count)] in host memory -> [(keys, counts, n_windows)]."""
    lib = load()
    keep = []
    arr = (_Job * max(len(jobs), 1))()
    for i, (b, o, k, m) in enumerate(jobs):
        b = _np(b, np.uint8)
        o = _np(o, np.uint64)
        keep.append((b, o))
        arr[i] = _Job(b.ctypes.data if b.size else None, o.ctypes.data, o.size - 1, k, m)
    outs = (_Result * max(len(jobs), 1))()
    rc = lib.turtle_count_batch(arr, len(jobs), ctypes.byref(params) if params else None, _stream_ptr(stream), outs)
    _check(rc, "turtle_count_batch")
    res = []
    for i, (_, _, k, _) in enumerate(jobs):
        r = _Result()
        ctypes.memmove(ctypes.byref(r), ctypes.byref(outs[i]), ctypes.sizeof(_Result))
        res.append(_take(lib, r, k))
    return res


class Server:
    """Served form: continuous batching of counting jobs admitted by device-memory footprint.

    Up to max_batch queued jobs with the same k and min_count share one batched run, and up to
    `executors` runs are on the device at once (each executor with its own context and stream).
    """

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_batch: int = 4,
                 params: Params | None = None, executors: int = 2):
        self._lib = load()
        self._h = _p()
        self._keep = {}
        _check(self._lib.turtle_server_create_ex(device, hbm_budget_bytes, max_batch, executors,
                                                 ctypes.byref(params) if params else None, ctypes.byref(self._h)),
               "turtle_server_create_ex")

    def submit(self, bases, offsets, k: int, min_count: int = 2) -> int:
        b = _np(bases, np.uint8)
        o = _np(offsets, np.uint64)
        job = _Job(b.ctypes.data if b.size else None, o.ctypes.data, o.size - 1, k, min_count)
        t = u64()
        _check(self._lib.turtle_submit(self._h, ctypes.byref(job), ctypes.byref(t)), "turtle_submit")
        self._keep[t.value] = (b, o, k)  # host reads must outlive the job
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(keys, counts, n_windows, JobTimes); raises TurtleError (TURTLE_E_TIMEOUT when not done yet)."""
        res = _Result()
        tm = JobTimes()
        rc = self._lib.turtle_poll(self._h, ticket, timeout_ms, ctypes.byref(res), ctypes.byref(tm))
        if rc == -5:
            raise TurtleError(rc, "turtle_poll")
        k = self._keep.pop(ticket, (None, None, 31))[2]
        if rc != 0:
            self._lib.turtle_result_free(ctypes.byref(res))
            _check(rc, "turtle_poll")
        keys, counts, nw = _take(self._lib, res, k)
        return keys, counts, nw, tm

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.turtle_server_stats_get(self._h, ctypes.byref(st)), "turtle_server_stats_get")
        return {f: int(getattr(st, f)) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            self._lib.turtle_server_destroy(self._h)
            self._h = _p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _CudaArray:
    """Zero-copy view of library-owned device memory (valid until the context's next call)."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _dptr(t) -> int:
    return t.data_ptr()


class Context:
    """A libturtle context on one device (owns scratch, the last device result and timing events)."""

    def __init__(self, device: int = 0):
        self._lib = load()
        self._h = _p()
        _check(self._lib.turtle_ctx_create(device, ctypes.byref(self._h)), "turtle_ctx_create")
        self.device = device

    def close(self):
        if self._h:
            self._lib.turtle_ctx_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ whole path
    def turtle_count(self, bases, offsets, k: int, min_count: int = 2, params: Params | None = None, stream=None):
        """Host-memory form on this context (turtle_ctx_count): NumPy in, (keys, counts, n_windows) out, as
        the module-level turtle_count; this context's stats() then include the host-side phases."""
        b = _np(bases, np.uint8)
        o = _np(offsets, np.uint64)
        reads = _Reads(b.ctypes.data if b.size else None, o.ctypes.data, o.size - 1)
        res = _Result()
        rc = self._lib.turtle_ctx_count(self._h, ctypes.byref(reads), k, min_count,
                                        ctypes.byref(params) if params else None, _stream_ptr(stream),
                                        ctypes.byref(res))
        _check(rc, "turtle_ctx_count")
        return _take(self._lib, res, k)

    def turtle_count_device(self, bases, offsets, k: int, min_count: int = 2, params: Params | None = None,
                            stream=None):
        """bases: CUDA uint8 tensor; offsets: CUDA int64/uint64 tensor (n_reads + 1).

        Returns (keys, counts, n_windows): torch CUDA views of context-owned memory,
        valid until this context's next call (clone them to keep them).
        """
        import torch
        assert bases.is_cuda and offsets.is_cuda and bases.dtype == torch.uint8
        assert offsets.dtype in (torch.int64, torch.uint64) and offsets.is_contiguous() and bases.is_contiguous()
        out = _DeviceResult()
        rc = self._lib.turtle_count_device(self._h, _dptr(bases), bases.numel(), _dptr(offsets), offsets.numel() - 1,
                                           k, min_count, ctypes.byref(params) if params else None,
                                           _stream_ptr(stream), ctypes.byref(out))
        _check(rc, "turtle_count_device")
        return self._views(out)

    def turtle_frequent_device(self, bases, offsets, k: int, params: Params | None = None, stream=None):
        """cTurtle on device-resident reads: (keys, n_windows), keys a torch CUDA view of context-owned
        memory valid until this context's next call."""
        import torch
        assert bases.is_cuda and offsets.is_cuda and bases.dtype == torch.uint8
        assert offsets.dtype in (torch.int64, torch.uint64) and offsets.is_contiguous() and bases.is_contiguous()
        out = _DeviceResult()
        rc = self._lib.turtle_frequent_device(self._h, _dptr(bases), bases.numel(), _dptr(offsets),
                                              offsets.numel() - 1, k, ctypes.byref(params) if params else None,
                                              _stream_ptr(stream), ctypes.byref(out))
        _check(rc, "turtle_frequent_device")
        n, w = int(out.n), int(out.key_words)
        if n == 0:
            return torch.zeros((0, 2) if w == 2 else (0,), dtype=torch.int64, device="cuda"), int(out.n_windows)
        keys = torch.as_tensor(_CudaArray(out.keys, (n, 2) if w == 2 else (n,), "<i8", self), device="cuda")
        return keys, int(out.n_windows)

    def _views(self, out):
        import torch
        n, w = int(out.n), int(out.key_words)
        if n == 0:
            return (torch.zeros((0, 2) if w == 2 else (0,), dtype=torch.int64, device="cuda"),
                    torch.zeros(0, dtype=torch.int32, device="cuda"), int(out.n_windows))
        keys = torch.as_tensor(_CudaArray(out.keys, (n, 2) if w == 2 else (n,), "<i8", self), device="cuda")
        counts = torch.as_tensor(_CudaArray(out.counts, (n,), "<i4", self), device="cuda")
        return keys, counts, int(out.n_windows)

    def stats(self) -> dict:
        st = Stats()
        _check(self._lib.turtle_ctx_stats(self._h, ctypes.byref(st)), "turtle_ctx_stats")
        return st.as_dict()

    def autotune(self, bases, offsets, k: int, min_count: int = 2, params: Params | None = None, stream=None):
        """turtle_autotune on device-resident reads: (tuned Params, TuneReport)."""
        best, rep = Params(), TuneReport()
        rc = self._lib.turtle_autotune(self._h, _dptr(bases), bases.numel(), _dptr(offsets), offsets.numel() - 1, k,
                                       min_count, ctypes.byref(params) if params else None, _stream_ptr(stream),
                                       ctypes.byref(best), ctypes.byref(rep))
        _check(rc, "turtle_autotune")
        return best, rep

    def trim(self):
        """Give back the device memory this context's pool keeps unused between calls."""
        self._lib.turtle_ctx_trim(self._h)

    def pool_bytes(self):
        """(bytes used by live buffers, bytes reserved) of this context's device memory pool."""
        used, reserved = u64(), u64()
        _check(self._lib.turtle_ctx_pool_bytes(self._h, ctypes.byref(used), ctypes.byref(reserved)),
               "turtle_ctx_pool_bytes")
        return int(used.value), int(reserved.value)

    # ------------------------------------------------------------ per-step entry points
    def turtle_extract(self, bases, offsets, k: int, stream=None):
        """(keys [n_bases(, 2)] int64 CUDA, valid bitmap [ceil(n/64)] int64 CUDA, n_windows)."""
        import torch
        n = bases.numel()
        w = 2 if k > 32 else 1
        keys = torch.empty((n, 2) if w == 2 else (n,), dtype=torch.int64, device=bases.device)
        valid = torch.zeros((n + 63) // 64, dtype=torch.int64, device=bases.device)
        nw = u64()
        rc = self._lib.turtle_extract(self._h, _dptr(bases), n, _dptr(offsets), offsets.numel() - 1, k,
                                      _stream_ptr(stream), _dptr(keys), _dptr(valid), ctypes.byref(nw))
        _check(rc, "turtle_extract")
        return keys, valid, int(nw.value)

    def turtle_filter(self, keys, filter_words, n_sectors: int, params: Params | None = None, set: bool = True,
                      stream=None):
        """Test(-and-set) keys (CUDA int64 [n] or [n, 2]) against filter_words (CUDA int64 [4*n_sectors])."""
        import torch
        n = keys.shape[0]
        w = 2 if keys.dim() == 2 else 1
        seen = torch.empty(n, dtype=torch.uint8, device=keys.device)
        rc = self._lib.turtle_filter(self._h, _dptr(keys), n, w, _dptr(filter_words), n_sectors,
                                     ctypes.byref(params) if params else None, 1 if set else 0, _dptr(seen),
                                     _stream_ptr(stream))
        _check(rc, "turtle_filter")
        return seen

    def turtle_sort_compact(self, keys, key_bits: int, stream=None):
        """Sort-and-compact CUDA keys: (unique keys, uint32 run lengths as int32) trimmed to n_unique."""
        import torch
        n = keys.shape[0]
        w = 2 if keys.dim() == 2 else 1
        uniq = torch.empty_like(keys)
        counts = torch.empty(n, dtype=torch.int32, device=keys.device)
        nu = u64()
        rc = self._lib.turtle_sort_compact(self._h, _dptr(keys), n, w, key_bits, _dptr(uniq), _dptr(counts),
                                           ctypes.byref(nu), _stream_ptr(stream))
        _check(rc, "turtle_sort_compact")
        return uniq[: nu.value], counts[: nu.value]
