"""Thin ctypes binding of the C ABI in ``include/ghn_knn.h`` and ``include/ghn_serve.h``.

Argument marshalling only: every step of index build and query runs in the
CUDA library ``_build/libghn_knn.so``.  There is no fallback: if the library
is missing, loading raises.  Arrays may be torch tensors (CUDA or CPU) or
numpy arrays; host arrays are staged to the GPU by the library itself.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

KNN_OK, KNN_EINVAL, KNN_ENOMEM, KNN_ECUDA, KNN_ELIMIT, KNN_ETIMEDOUT = 0, 1, 2, 3, 4, 5
KNN_NONE, KNN_VOTE, KNN_MEAN, KNN_MEDIAN = -1, 0, 1, 2
KNN_TABLE_AUTO, KNN_TABLE_DENSE, KNN_TABLE_HASH = 0, 1, 2
KNN_QUERY_CHECKED, KNN_QUERY_SORTED, KNN_QUERY_EXACT = 1, 2, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libghn_knn.so")

_lock = threading.Lock()
_lib = None


class KnnError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"[status {code}] {message}")
        self.code = code


class knn_index_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("table", ctypes.c_int32),
                ("cell_width", ctypes.c_float), ("origin", ctypes.c_float * 8),
                ("extent", ctypes.c_int64 * 8), ("num_cells", ctypes.c_int64),
                ("table_slots", ctypes.c_int64), ("row_floats", ctypes.c_int32),
                ("has_labels", ctypes.c_int32)]


EXPORTED = ["knn_batch_build", "knn_batch_info", "knn_batch_query", "knn_batch_plan",
            "knn_batch_run", "knn_plan_free", "knn_batch_free",
            "knn_build", "knn_build_grid", "knn_measure_cells", "knn_index_grid", "knn_query", "knn_query_stats", "knn_query_noalloc", "knn_index_info",
            "knn_index_export", "knn_index_set_deferral", "knn_batch_set_deferral",
            "knn_timing_enable", "knn_timing_read", "knn_kernel_launches", "knn_free",
            "knn_last_error", "knn_abi_version",
            "knn_server_create", "knn_server_build", "knn_server_drop", "knn_server_submit",
            "knn_server_submit_many",
            "knn_server_wait", "knn_server_test", "knn_server_stats", "knn_server_clock_ns",
            "knn_server_build_bytes", "knn_server_index", "knn_server_destroy"]


class knn_server_config(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("max_batch_queries", ctypes.c_int64),
                ("max_batch_outputs", ctypes.c_int64), ("max_batch_requests", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("device", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class knn_ticket_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("index_id", ctypes.c_int64), ("batch", ctypes.c_int64),
                ("t_submit_ns", ctypes.c_int64), ("t_dispatch_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class knn_server_stats_t(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "batches", "requests_done", "queries_done", "builds_done", "drops_done", "indexes",
        "resident_bytes", "reserved_bytes", "buffer_bytes", "budget_bytes", "queued_requests",
        "waiting_builds", "inflight_batches", "max_batch_requests_seen",
        "max_batch_queries_seen", "pack_ns", "wait_ns", "scatter_ns")]


def library(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built).  GHN_LIB may
    name another build of it (for comparing builds)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or os.environ.get("GHN_LIB") or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing "
                               "(run __graft_entry__.build() or build_ext.build())")
        lib = ctypes.CDLL(p)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.knn_build.argtypes = [vp, vp, i64, i32, ctypes.c_float, i32, vp, ctypes.POINTER(vp)]
        lib.knn_build.restype = i32
        lib.knn_build_grid.argtypes = [vp, vp, i64, i32, vp, vp, i32, vp, ctypes.POINTER(vp)]
        lib.knn_build_grid.restype = i32
        lib.knn_measure_cells.argtypes = [vp, i64, i32, vp, vp, vp]
        lib.knn_measure_cells.restype = i32
        lib.knn_index_grid.argtypes = [vp, vp, vp]
        lib.knn_index_grid.restype = i32
        lib.knn_query.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, i32, vp]
        lib.knn_query.restype = i32
        lib.knn_query_stats.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp]
        lib.knn_query_stats.restype = i32
        lib.knn_query_noalloc.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, i32, vp]
        lib.knn_query_noalloc.restype = i32
        lib.knn_index_info.argtypes = [vp, ctypes.POINTER(knn_index_info_t)]
        lib.knn_index_info.restype = i32
        lib.knn_index_export.argtypes = [vp, vp, vp, vp]
        lib.knn_index_export.restype = i32
        lib.knn_index_set_deferral.argtypes = [vp, i64, i64]
        lib.knn_index_set_deferral.restype = i32
        lib.knn_batch_set_deferral.argtypes = [vp, i32, i64, i64]
        lib.knn_batch_set_deferral.restype = i32
        lib.knn_free.argtypes = [vp]
        lib.knn_free.restype = None
        lib.knn_last_error.argtypes = []
        lib.knn_last_error.restype = ctypes.c_char_p
        lib.knn_abi_version.argtypes = []
        lib.knn_abi_version.restype = i32
        lib.knn_timing_enable.argtypes = [i32]
        lib.knn_timing_enable.restype = i32
        lib.knn_timing_read.argtypes = [ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.POINTER(ctypes.c_float), i32]
        lib.knn_timing_read.restype = i32
        lib.knn_kernel_launches.argtypes = []
        lib.knn_kernel_launches.restype = i64
        pp = ctypes.POINTER(vp)
        lib.knn_batch_build.argtypes = [i32, pp, pp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32), vp,
                                        ctypes.POINTER(vp)]
        lib.knn_batch_build.restype = i32
        lib.knn_batch_info.argtypes = [vp, i32, ctypes.POINTER(knn_index_info_t)]
        lib.knn_batch_info.restype = i32
        lib.knn_batch_query.argtypes = [vp, pp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                        ctypes.POINTER(i32), pp, pp, pp, i32, vp]
        lib.knn_batch_query.restype = i32
        lib.knn_batch_plan.argtypes = [vp, pp, ctypes.POINTER(i64), ctypes.POINTER(i32),
                                       ctypes.POINTER(i32), pp, pp, pp, ctypes.POINTER(vp)]
        lib.knn_batch_plan.restype = i32
        lib.knn_batch_run.argtypes = [vp, i32, vp]
        lib.knn_batch_run.restype = i32
        lib.knn_plan_free.argtypes = [vp]
        lib.knn_plan_free.restype = None
        lib.knn_batch_free.argtypes = [vp]
        lib.knn_batch_free.restype = None
        pi64 = ctypes.POINTER(i64)
        lib.knn_server_create.argtypes = [ctypes.POINTER(knn_server_config), ctypes.POINTER(vp)]
        lib.knn_server_create.restype = i32
        lib.knn_server_build.argtypes = [vp, vp, vp, i64, i32, ctypes.c_float, i32, pi64, pi64]
        lib.knn_server_build.restype = i32
        lib.knn_server_drop.argtypes = [vp, i64, pi64]
        lib.knn_server_drop.restype = i32
        lib.knn_server_submit.argtypes = [vp, i64, vp, i64, i32, i32, vp, vp, vp, i32, pi64]
        lib.knn_server_submit.restype = i32
        lib.knn_server_submit_many.argtypes = [vp, i32, pi64, pp, pi64, ctypes.POINTER(i32),
                                               ctypes.POINTER(i32), pp, pp, pp,
                                               ctypes.POINTER(i32), pi64]
        lib.knn_server_submit_many.restype = i32
        lib.knn_server_wait.argtypes = [vp, i64, i64, ctypes.POINTER(knn_ticket_info)]
        lib.knn_server_wait.restype = i32
        lib.knn_server_test.argtypes = [vp, i64, ctypes.POINTER(i32),
                                        ctypes.POINTER(knn_ticket_info)]
        lib.knn_server_test.restype = i32
        lib.knn_server_stats.argtypes = [vp, ctypes.POINTER(knn_server_stats_t)]
        lib.knn_server_stats.restype = i32
        lib.knn_server_clock_ns.argtypes = []
        lib.knn_server_clock_ns.restype = i64
        lib.knn_server_index.argtypes = [vp, i64, ctypes.POINTER(vp)]
        lib.knn_server_index.restype = i32
        lib.knn_server_build_bytes.argtypes = [i64, i32, i32]
        lib.knn_server_build_bytes.restype = i64
        lib.knn_server_destroy.argtypes = [vp]
        lib.knn_server_destroy.restype = None
        _lib = lib
        return lib


def _check(code: int):
    if code != KNN_OK:
        raise KnnError(code, library().knn_last_error().decode(errors="replace"))


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(address, keepalive) of a contiguous torch tensor or numpy array, or (None, None)."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a)
    return arr.ctypes.data, arr


def _stream(stream, *arrays):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _check_f32(a, name):
    dt = str(a.dtype)
    if not dt.endswith("float32"):
        raise ValueError(f"{name} must be float32, got {dt}")


class Index:
    """A built GHN index (device memory owned by the library)."""

    def __init__(self, handle: ctypes.c_void_p, n: int, d: int):
        self._h = handle
        self.n = n
        self.d = d

    @property
    def handle(self) -> int:
        return self._h.value

    def info(self) -> knn_index_info_t:
        out = knn_index_info_t()
        _check(library().knn_index_info(self._h, ctypes.byref(out)))
        return out

    def grid(self):
        """(widths float32[d], splits int64[d]) the index was built with (splits 0: none)."""
        w = np.zeros(self.d, np.float32)
        sp = np.zeros(self.d, np.int64)
        _check(library().knn_index_grid(self._h, w.ctypes.data, sp.ctypes.data))
        return w, sp

    def export(self):
        """(cell_keys uint64, cell_start uint32, rows int32) as numpy arrays."""
        inf = self.info()
        u = int(inf.num_cells)
        keys = np.zeros(u, np.uint64)
        starts = np.zeros(u + 1, np.uint32)
        rows = np.zeros(self.n, np.int32)
        _check(library().knn_index_export(self._h, keys.ctypes.data, starts.ctypes.data,
                                          rows.ctypes.data))
        return keys, starts, rows

    def query(self, queries, k: int, mode: int = KNN_NONE, flags: int = 0, stream=None,
              ids=None, dist2=None, pred=None, want_dist2: bool = True):
        return knn_query(self, queries, k, mode, flags=flags, stream=stream, ids=ids,
                         dist2=dist2, pred=pred, want_dist2=want_dist2)

    def query_stats(self, queries, k: int, stream=None):
        return knn_query_stats(self, queries, k, stream=stream)

    def set_deferral(self, heavy_rows: int = 0, heavy_cands: int = 0):
        """Thresholds for handing heavy queries to the cooperative kernel
        (0: library default, < 0: never); results do not depend on them."""
        _check(library().knn_index_set_deferral(self._h, int(heavy_rows), int(heavy_cands)))

    def free(self):
        if self._h is not None and self._h.value:
            library().knn_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def knn_build(points, labels=None, cell_width: float = 1.0, table: int = KNN_TABLE_AUTO,
              stream=None) -> Index:
    """Cell sampling (Sec. III.A): returns an Index over n x d float32 points."""
    if points.ndim != 2:
        raise ValueError("points must be n x d")
    _check_f32(points, "points")
    n, d = int(points.shape[0]), int(points.shape[1])
    pp, keep_p = _ptr(points)
    lp, keep_l = _ptr(labels)
    if labels is not None and (labels.shape[0] != n or np.dtype(str(labels.dtype).split(".")[-1]).itemsize != 4):
        raise ValueError("labels must be n 32-bit values")
    h = ctypes.c_void_p()
    _check(library().knn_build(pp, lp, n, d, ctypes.c_float(float(np.float32(cell_width))),
                               table, _stream(stream, points, labels), ctypes.byref(h)))
    del keep_p, keep_l
    return Index(h, n, d)


def knn_build_grid(points, labels=None, cell_widths=None, splits=None,
                   table: int = KNN_TABLE_AUTO, stream=None) -> Index:
    """Cell sampling with one cell measurement per dimension (and optional split counts)."""
    if points.ndim != 2:
        raise ValueError("points must be n x d")
    _check_f32(points, "points")
    n, d = int(points.shape[0]), int(points.shape[1])
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(cell_widths, np.float32), (d,)),
                             np.float32)
    sp = None if splits is None else np.ascontiguousarray(splits, np.int64)
    if sp is not None and sp.shape != (d,):
        raise ValueError("splits must have d entries")
    pp, keep_p = _ptr(points)
    lp, keep_l = _ptr(labels)
    h = ctypes.c_void_p()
    _check(library().knn_build_grid(pp, lp, n, d, w.ctypes.data,
                                    sp.ctypes.data if sp is not None else None, table,
                                    _stream(stream, points, labels), ctypes.byref(h)))
    del keep_p, keep_l
    return Index(h, n, d)


def knn_measure_cells(points, stream=None):
    """The paper's cell measurement (Sec. III.A) on the GPU: (splits int64[d], widths float32[d])."""
    if points.ndim != 2:
        raise ValueError("points must be n x d")
    _check_f32(points, "points")
    n, d = int(points.shape[0]), int(points.shape[1])
    splits = np.zeros(d, np.int64)
    widths = np.zeros(d, np.float32)
    pp, keep = _ptr(points)
    _check(library().knn_measure_cells(pp, n, d, splits.ctypes.data, widths.ctypes.data,
                                       _stream(stream, points)))
    del keep
    return splits, widths


def _alloc_like(ref, shape, dtype_name):
    if ref is not None and _is_torch(ref):
        import torch
        return torch.empty(shape, dtype=getattr(torch, dtype_name), device=ref.device)
    return np.empty(shape, dtype=dtype_name)


def knn_query(index: Index, queries, k: int, mode: int = KNN_NONE, flags: int = 0, stream=None,
              ids=None, dist2=None, pred=None, want_dist2: bool = True):
    """Exploration + prediction (Sec. III.B, Sec. I): returns (ids, dist2, pred)."""
    if queries.ndim != 2 or queries.shape[1] != index.d:
        raise ValueError("queries must be m x d")
    _check_f32(queries, "queries")
    m = int(queries.shape[0])
    if ids is None:
        ids = _alloc_like(queries, (m, k), "int32")
    if dist2 is None and want_dist2:
        dist2 = _alloc_like(queries, (m, k), "float32")
    if pred is None and mode >= 0:
        pred = _alloc_like(queries, (m,), "int32" if mode == KNN_VOTE else "float32")
    qp, kq = _ptr(queries)
    ip, ki = _ptr(ids)
    dp, kd = _ptr(dist2)
    pp, kp = _ptr(pred)
    _check(library().knn_query(index._h, qp, m, k, mode, ip, dp, pp, flags,
                               _stream(stream, queries, ids)))
    del kq, ki, kd, kp
    return ids, dist2, pred


def knn_query_stats(index: Index, queries, k: int, stream=None):
    """Walk without skipping; returns (ids, dist2, stats m x 3 int64)."""
    m = int(queries.shape[0])
    ids = _alloc_like(queries, (m, k), "int32")
    dist2 = _alloc_like(queries, (m, k), "float32")
    stats = _alloc_like(queries, (m, 3), "int64")
    qp, kq = _ptr(queries)
    ip, ki = _ptr(ids)
    dp, kd = _ptr(dist2)
    sp, ks = _ptr(stats)
    _check(library().knn_query_stats(index._h, qp, m, k, ip, dp, sp,
                                     _stream(stream, queries, ids)))
    del kq, ki, kd, ks
    return ids, dist2, stats


def knn_query_noalloc(index: Index, queries, k: int, mode: int, ids, dist2=None, pred=None,
                      flags: int = 0, stream=None):
    """knn_query into caller-allocated device tensors, allocating nothing.

    For callers that cannot allocate device memory while they query; the
    library's fixed scratch array is used instead (m <= 1048576, device
    buffers only, calls must not overlap on the GPU).
    """
    m = int(queries.shape[0])
    qp, kq = _ptr(queries)
    ip, ki = _ptr(ids)
    dp, kd = _ptr(dist2)
    pp, kp = _ptr(pred)
    _check(library().knn_query_noalloc(index._h, qp, m, k, mode, ip, dp, pp, flags,
                                       _stream(stream, queries, ids)))
    del kq, ki, kd, kp
    return ids, dist2, pred


def _ptr_array(items):
    """A ctypes array of the addresses of tensors (None -> NULL) and their keepalives."""
    arr = (ctypes.c_void_p * len(items))()
    keep = []
    for i, a in enumerate(items):
        p, k = _ptr(a)
        arr[i] = p
        keep.append(k)
    return arr, keep


class Batch:
    """A batch of independent indexes built in one pass (knn_batch_build)."""

    def __init__(self, handle, ns, ds):
        self._h = handle
        self.ns = list(ns)
        self.ds = list(ds)
        self.count = len(self.ns)

    def info(self, i: int) -> knn_index_info_t:
        out = knn_index_info_t()
        _check(library().knn_batch_info(self._h, i, ctypes.byref(out)))
        return out

    def set_deferral(self, i: int, heavy_rows: int = 0, heavy_cands: int = 0):
        """Deferral thresholds of index i (as Index.set_deferral)."""
        _check(library().knn_batch_set_deferral(self._h, int(i), int(heavy_rows),
                                                int(heavy_cands)))

    def _outputs(self, queries, ks, modes):
        ids, d2, pred = [], [], []
        for q, k, mode in zip(queries, ks, modes):
            m = int(q.shape[0])
            ids.append(_alloc_like(q, (m, k), "int32"))
            d2.append(_alloc_like(q, (m, k), "float32"))
            pred.append(None if mode < 0 else
                        _alloc_like(q, (m,), "int32" if mode == KNN_VOTE else "float32"))
        return ids, d2, pred

    def _arrays(self, queries, ks, modes, ids, d2, pred):
        if not (len(queries) == len(ks) == len(modes) == self.count):
            raise ValueError("one query set, k and mode per index")
        m = (ctypes.c_int64 * self.count)(*[int(q.shape[0]) for q in queries])
        k = (ctypes.c_int32 * self.count)(*ks)
        md = (ctypes.c_int32 * self.count)(*modes)
        qa, kq = _ptr_array(queries)
        ia, ki = _ptr_array(ids)
        da, kd = _ptr_array(d2)
        pa, kp = _ptr_array(pred)
        return (m, k, md, qa, ia, da, pa), (kq, ki, kd, kp)

    def query(self, queries, ks, modes, flags: int = 0, stream=None, out=None):
        """Query every index; returns lists (ids, dist2, pred) with one entry per index.

        Queries and outputs may be host arrays or device tensors; `out`, if
        given, is (ids, dist2, pred) lists of caller buffers to fill."""
        ids, d2, pred = self._outputs(queries, ks, modes) if out is None else out
        (m, k, md, qa, ia, da, pa), keep = self._arrays(queries, ks, modes, ids, d2, pred)
        _check(library().knn_batch_query(self._h, qa, m, k, md, ia, da, pa, flags,
                                         _stream(stream, *queries)))
        del keep
        return ids, d2, pred

    def plan(self, queries, ks, modes):
        """Capture the query of these buffers in a CUDA graph; returns (Plan, ids, dist2, pred)."""
        ids, d2, pred = self._outputs(queries, ks, modes)
        (m, k, md, qa, ia, da, pa), keep = self._arrays(queries, ks, modes, ids, d2, pred)
        h = ctypes.c_void_p()
        _check(library().knn_batch_plan(self._h, qa, m, k, md, ia, da, pa, ctypes.byref(h)))
        return Plan(h, (queries, ids, d2, pred, keep)), ids, d2, pred

    def free(self):
        if self._h is not None and self._h.value:
            library().knn_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Plan:
    """A batch query captured in a CUDA graph (knn_batch_plan); run() replays it."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep  # the buffers the graph reads and writes

    def run(self, flags: int = 0, stream=None):
        _check(library().knn_batch_run(self._h, flags, _stream(stream, *self._keep[0])))

    def free(self):
        if self._h is not None and self._h.value:
            library().knn_plan_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def knn_batch_build(points, labels, widths, tables=None, stream=None) -> Batch:
    """Build one index per entry of `points` (lists; labels entries may be None)."""
    count = len(points)
    for p in points:
        if p.ndim != 2:
            raise ValueError("points must be n x d")
        _check_f32(p, "points")
    ns = [int(p.shape[0]) for p in points]
    ds = [int(p.shape[1]) for p in points]
    pa, kp = _ptr_array(points)
    la, kl = _ptr_array(labels if labels is not None else [None] * count)
    n = (ctypes.c_int64 * count)(*ns)
    d = (ctypes.c_int32 * count)(*ds)
    w = (ctypes.c_float * count)(*[float(np.float32(x)) for x in widths])
    t = None if tables is None else (ctypes.c_int32 * count)(*tables)
    h = ctypes.c_void_p()
    _check(library().knn_batch_build(count, pa, la, n, d, w, t, _stream(stream, *points),
                                     ctypes.byref(h)))
    del kp, kl
    return Batch(h, ns, ds)


def knn_free(index: Index):
    index.free()


def knn_timing_enable(on: bool = True):
    _check(library().knn_timing_enable(1 if on else 0))


def knn_timing_read() -> list[tuple[str, float]]:
    """Phases of this thread's oldest unread call (of its last 32, while timing
    is on): [(name, device ms)], or [] when none is unread."""
    names = (ctypes.c_char_p * 40)()
    ms = (ctypes.c_float * 40)()
    cnt = library().knn_timing_read(names, ms, 40)
    return [(names[i].decode(), float(ms[i])) for i in range(min(cnt, 40))]


def knn_kernel_launches() -> int:
    return int(library().knn_kernel_launches())


def knn_last_error() -> str:
    return library().knn_last_error().decode(errors="replace")


# ---- serving engine (include/ghn_serve.h) ----

class Server:
    """A serving engine: resident indexes, memory-admitted builds, continuous batching.

    Requests return tickets at once; ``wait`` returns a ticket's outcome.  The
    host arrays of a request (numpy) are kept alive here until its ticket is
    waited for.
    """

    def __init__(self, memory_budget: int = 0, max_batch_queries: int = 0,
                 max_batch_outputs: int = 0, max_batch_requests: int = 0, max_inflight: int = 0,
                 device: int = 0):
        cfg = knn_server_config(memory_budget, max_batch_queries, max_batch_outputs,
                                max_batch_requests, max_inflight, device, 0)
        h = ctypes.c_void_p()
        _check(library().knn_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}  # ticket -> arrays the request borrows or fills
        self._klock = threading.Lock()

    def build(self, points, labels=None, cell_width: float = 1.0, table: int = KNN_TABLE_AUTO):
        """Request a new index; returns (index_id, ticket)."""
        n, d = int(points.shape[0]), int(points.shape[1])
        pp, kp = _ptr(points)
        lp, kl = _ptr(labels)
        iid, t = ctypes.c_int64(), ctypes.c_int64()
        _check(library().knn_server_build(self._h, pp, lp, n, d,
                                          ctypes.c_float(float(np.float32(cell_width))), table,
                                          ctypes.byref(iid), ctypes.byref(t)))
        with self._klock:
            self._keep[t.value] = (points, labels, kp, kl)
        return iid.value, t.value

    def drop(self, index_id: int) -> int:
        t = ctypes.c_int64()
        _check(library().knn_server_drop(self._h, index_id, ctypes.byref(t)))
        return t.value

    def submit(self, index_id: int, queries: np.ndarray, k: int, mode: int = KNN_NONE,
               want_dist2: bool = True, flags: int = 0):
        """Queue a query request (host arrays); returns (ticket, ids, dist2, pred).

        flags: 0 or KNN_QUERY_EXACT (the certified stop for this request).
        """
        q = np.ascontiguousarray(queries, np.float32)
        m = int(q.shape[0])
        ids = np.empty((m, k), np.int32)
        d2 = np.empty((m, k), np.float32) if want_dist2 else None
        pred = None
        if mode >= 0:
            pred = np.empty(m, np.int32 if mode == KNN_VOTE else np.float32)
        t = ctypes.c_int64()
        _check(library().knn_server_submit(
            self._h, index_id, q.ctypes.data, m, k, mode, ids.ctypes.data,
            d2.ctypes.data if d2 is not None else None,
            pred.ctypes.data if pred is not None else None, flags, ctypes.byref(t)))
        with self._klock:
            self._keep[t.value] = (q, ids, d2, pred)
        return t.value, ids, d2, pred

    def submit_many(self, requests, want_dist2: bool = True):
        """Queue many requests in one call: requests is a list of
        (index_id, queries, k, mode[, flags]); returns [(ticket, ids, dist2, pred)]."""
        n = len(requests)
        c = ctypes
        iid = (c.c_int64 * n)()
        qp = (c.c_void_p * n)()
        mm = (c.c_int64 * n)()
        kk = (c.c_int32 * n)()
        md = (c.c_int32 * n)()
        ip = (c.c_void_p * n)()
        dp = (c.c_void_p * n)()
        pp_ = (c.c_void_p * n)()
        fl = (c.c_int32 * n)()
        tk = (c.c_int64 * n)()
        out, keep = [], []
        for i, r in enumerate(requests):
            index_id, queries, k, mode = r[:4]
            q = np.ascontiguousarray(queries, np.float32)
            m = int(q.shape[0])
            ids = np.empty((m, k), np.int32)
            d2 = np.empty((m, k), np.float32) if want_dist2 else None
            pred = None
            if mode >= 0:
                pred = np.empty(m, np.int32 if mode == KNN_VOTE else np.float32)
            iid[i], qp[i], mm[i], kk[i], md[i] = index_id, q.ctypes.data, m, k, mode
            ip[i] = ids.ctypes.data
            dp[i] = d2.ctypes.data if d2 is not None else None
            pp_[i] = pred.ctypes.data if pred is not None else None
            fl[i] = r[4] if len(r) > 4 else 0
            out.append([None, ids, d2, pred])
            keep.append(q)
        _check(library().knn_server_submit_many(self._h, n, iid, qp, mm, kk, md, ip, dp, pp_, fl,
                                                tk))
        with self._klock:
            for i in range(n):
                out[i][0] = tk[i]
                self._keep[tk[i]] = (keep[i], out[i][1], out[i][2], out[i][3])
        return [tuple(o) for o in out]

    def wait(self, ticket: int, timeout_us: int = -1):
        """Outcome of a ticket (knn_ticket_info), or None if the timeout ran out."""
        info = knn_ticket_info()
        rc = library().knn_server_wait(self._h, ticket, timeout_us, ctypes.byref(info))
        if rc == KNN_ETIMEDOUT:
            return None
        _check(rc)
        with self._klock:
            self._keep.pop(ticket, None)
        return info

    def test(self, ticket: int):
        info = knn_ticket_info()
        done = ctypes.c_int32()
        _check(library().knn_server_test(self._h, ticket, ctypes.byref(done), ctypes.byref(info)))
        if not done.value:
            return None
        with self._klock:
            self._keep.pop(ticket, None)
        return info

    def index(self, index_id: int) -> "Index":
        """The resident index behind an id, for plain queries (borrowed: never free it)."""
        h = ctypes.c_void_p()
        _check(library().knn_server_index(self._h, index_id, ctypes.byref(h)))
        info = knn_index_info_t()
        _check(library().knn_index_info(h, ctypes.byref(info)))
        return _Borrowed(h, int(info.n), int(info.d))

    def stats(self) -> knn_server_stats_t:
        s = knn_server_stats_t()
        _check(library().knn_server_stats(self._h, ctypes.byref(s)))
        return s

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            library().knn_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Borrowed(Index):
    """An index owned by a server: queries work, freeing is the server's job."""

    def free(self):
        self._h = ctypes.c_void_p()

    def __del__(self):
        pass


def knn_server_build_bytes(n: int, d: int, labels: bool) -> int:
    """Bytes a build of n points in d dimensions is admitted with (its footprint bound)."""
    return int(library().knn_server_build_bytes(n, d, int(bool(labels))))


def knn_server_clock_ns() -> int:
    """The serving engine's clock (CLOCK_MONOTONIC, ns); equals time.monotonic_ns()."""
    return int(library().knn_server_clock_ns())
