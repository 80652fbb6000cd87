"""ctypes front end of the C oracle (``ghn_oracle.c``).

Test infrastructure only: the product path never imports this module.  The C
file is compiled with ``-O2 -ffp-contract=off`` (no fused multiply-add, so that
squared distances are the dimension-order sums of rounded products the method
is checked on) and no fast-math.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ghn_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libghn_oracle.so")

_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def compile_c(src: str, out: str) -> None:
    """gcc, plain C11, no contraction into fused multiply-add, no fast-math."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build_library(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libghn_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    compile_c(_SRC, _LIB_PATH)
    return _LIB_PATH


def library() -> ctypes.CDLL:
    """The oracle library (GHN_ORACLE_LIB may name another build of it, for the mutation test)."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(os.environ.get("GHN_ORACLE_LIB") or build_library())
            vp = ctypes.c_void_p
            lib.oracle_build.argtypes = [_f32p, _u32p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_float, ctypes.POINTER(vp)]
            lib.oracle_build.restype = ctypes.c_int
            lib.oracle_build_grid.argtypes = [_f32p, _u32p, ctypes.c_int64, ctypes.c_int32,
                                              _f32p, _i64p, ctypes.POINTER(vp)]
            lib.oracle_build_grid.restype = ctypes.c_int
            lib.oracle_measure.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, _i64p, _f32p]
            lib.oracle_measure.restype = ctypes.c_int
            lib.oracle_query_rule.argtypes = [vp, _f32p, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, _i32p, _f32p, vp,
                                              _i64p]
            lib.oracle_query_rule.restype = ctypes.c_int
            lib.oracle_free.argtypes = [vp]
            lib.oracle_free.restype = None
            lib.oracle_query.argtypes = [vp, _f32p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_int32, _i32p, _f32p, vp, _i64p]
            lib.oracle_query.restype = ctypes.c_int
            lib.oracle_query_ex.argtypes = [vp, _f32p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, _i32p, _f32p, vp, _i64p]
            lib.oracle_query_ex.restype = ctypes.c_int
            lib.oracle_brute.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32, _f32p,
                                         ctypes.c_int64, ctypes.c_int32, _i32p, _f32p]
            lib.oracle_brute.restype = ctypes.c_int
            lib.oracle_shell_count.argtypes = [ctypes.c_int32, ctypes.c_int64]
            lib.oracle_shell_count.restype = ctypes.c_int64
            lib.oracle_num_cells.argtypes = [vp]
            lib.oracle_num_cells.restype = ctypes.c_int64
            lib.oracle_origin.argtypes = [vp, _f32p, _i64p]
            lib.oracle_origin.restype = None
            lib.oracle_cells.argtypes = [vp, _i64p, _i64p, _i32p]
            lib.oracle_cells.restype = None
            lib.oracle_cells_of.argtypes = [vp, _f32p, ctypes.c_int64, ctypes.c_int32, _i64p]
            lib.oracle_cells_of.restype = None
            lib.oracle_count_cells.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_float]
            lib.oracle_count_cells.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


RULE_NONE, RULE_PAPER, RULE_EXACT = 0, 1, 2


def measure_cells(points):
    """The paper's cell measurement (Sec. III.A): (splits int64[d], widths float32[d])."""
    pts = _f32(points)
    n, d = pts.shape
    splits = np.zeros(d, np.int64)
    widths = np.zeros(d, np.float32)
    rc = library().oracle_measure(_ptr(pts, _f32p), n, d, _ptr(splits, _i64p),
                                  _ptr(widths, _f32p))
    if rc != 0:
        raise ValueError(f"oracle_measure failed with code {rc}")
    return splits, widths


class Grid:
    """The oracle's grid (Algorithm 1) over training points with 32-bit outputs.

    w: one width, or d widths (one per dimension); splits: d split counts
    (training cells clamped to split - 1, the grid of the cell measurement)
    or None.
    """

    def __init__(self, points, labels, w, splits=None):
        lib = library()
        pts = _f32(points)
        if pts.ndim != 2:
            raise ValueError("points must be n x d")
        self.n, self.d = pts.shape
        wv = np.asarray(w, np.float32)
        self.widths = np.ascontiguousarray(np.broadcast_to(wv, (self.d,)) if wv.ndim == 0 else wv,
                                           np.float32)
        if self.widths.shape != (self.d,):
            raise ValueError("w must be a scalar or d widths")
        self.w = self.widths[0] if wv.ndim == 0 else self.widths
        self.splits = None if splits is None else np.ascontiguousarray(splits, np.int64)
        self._labels = None
        lab_p = None
        if labels is not None:
            lab = np.ascontiguousarray(labels)
            if lab.dtype.itemsize != 4 or lab.shape != (self.n,):
                raise ValueError("labels must be n 32-bit values")
            self._labels = lab
            lab_p = _ptr(lab.view(np.uint32), _u32p)
        h = ctypes.c_void_p()
        rc = lib.oracle_build_grid(_ptr(pts, _f32p), lab_p, self.n, self.d,
                                   _ptr(self.widths, _f32p),
                                   _ptr(self.splits, _i64p) if self.splits is not None else None,
                                   ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle_build failed with code {rc}")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.oracle_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_cells(self) -> int:
        return int(self._lib.oracle_num_cells(self._h))

    def origin(self):
        o = np.zeros(self.d, np.float32)
        cmax = np.zeros(self.d, np.int64)
        self._lib.oracle_origin(self._h, _ptr(o, _f32p), _ptr(cmax, _i64p))
        return o, cmax

    def cells(self):
        """(coords U x d int64, counts U int64, members list of int32 arrays) in creation order."""
        u = self.num_cells
        coords = np.zeros((u, self.d), np.int64)
        counts = np.zeros(u, np.int64)
        members = np.zeros(self.n, np.int32)
        self._lib.oracle_cells(self._h, _ptr(coords, _i64p), _ptr(counts, _i64p),
                               _ptr(members, _i32p))
        offs = np.concatenate([[0], np.cumsum(counts)])
        return coords, counts, [members[offs[e]:offs[e + 1]] for e in range(u)]

    def cells_of(self, pts, as_query: bool = False) -> np.ndarray:
        p = _f32(pts).reshape(-1, self.d)
        c = np.zeros(p.shape, np.int64)
        self._lib.oracle_cells_of(self._h, _ptr(p, _f32p), p.shape[0], int(as_query),
                                  _ptr(c, _i64p))
        return c

    def query(self, queries, k: int, mode: int = -1, stats: bool = False, rule: int = RULE_PAPER):
        """Neighbours of each query: (ids m x k, dist2 m x k, pred m or None[, stats m x 3]).

        mode: 0 vote (int32 outputs), 1 mean, 2 median (float outputs), -1 none.
        rule: RULE_PAPER (Sec. III.B), RULE_EXACT (certified stop), RULE_NONE.
        """
        q = _f32(queries).reshape(-1, self.d)
        m = q.shape[0]
        ids = np.zeros((m, k), np.int32)
        d2 = np.zeros((m, k), np.float32)
        pred = None
        if mode == 0:
            pred = np.zeros(m, np.int32)
        elif mode in (1, 2):
            pred = np.zeros(m, np.float32)
        st = np.zeros((m, 3), np.int64) if stats else None
        rc = self._lib.oracle_query_rule(self._h, _ptr(q, _f32p), m, k, mode, rule,
                                         _ptr(ids, _i32p), _ptr(d2, _f32p),
                                         pred.ctypes.data_as(ctypes.c_void_p)
                                         if pred is not None else None,
                                         _ptr(st, _i64p) if st is not None else None)
        if rc != 0:
            raise ValueError(f"oracle_query failed with code {rc}")
        return (ids, d2, pred, st) if stats else (ids, d2, pred)

    def query_one(self, q, k: int, mode: int = -1, stop_rule: bool = True):
        qq = _f32(q).reshape(self.d)
        ids = np.zeros(k, np.int32)
        d2 = np.zeros(k, np.float32)
        pred = np.zeros(1, np.int32 if mode == 0 else np.float32)
        st = np.zeros(3, np.int64)
        rc = self._lib.oracle_query_ex(self._h, _ptr(qq, _f32p), k, mode, int(stop_rule),
                                       _ptr(ids, _i32p), _ptr(d2, _f32p),
                                       pred.ctypes.data_as(ctypes.c_void_p) if mode >= 0
                                       else None, _ptr(st, _i64p))
        if rc != 0:
            raise ValueError(f"oracle_query_ex failed with code {rc}")
        return ids, d2, (pred[0] if mode >= 0 else None), st


def brute_force(points, queries, k: int):
    """Original KNN: exhaustive scan + sort by (dist2, index)."""
    lib = library()
    pts = _f32(points)
    n, d = pts.shape
    q = _f32(queries).reshape(-1, d)
    m = q.shape[0]
    ids = np.zeros((m, k), np.int32)
    d2 = np.zeros((m, k), np.float32)
    rc = lib.oracle_brute(_ptr(pts, _f32p), n, d, _ptr(q, _f32p), m, k, _ptr(ids, _i32p),
                          _ptr(d2, _f32p))
    if rc != 0:
        raise ValueError(f"oracle_brute failed with code {rc}")
    return ids, d2


def shell_count(d: int, layer: int) -> int:
    """Cells on layer `layer` of an unbounded d-dim grid, by the oracle's enumerator."""
    return int(library().oracle_shell_count(d, layer))


def count_cells(points, w: float) -> int:
    """Occupied cells of the grid of width w (used by the cell-width search)."""
    pts = _f32(points)
    n, d = pts.shape
    u = library().oracle_count_cells(_ptr(pts, _f32p), n, d, ctypes.c_float(np.float32(w)))
    if u < 0:
        raise ValueError("count_cells failed")
    return int(u)


def recall(grid: "Grid", points, queries, k: int):
    """Recall of the paper's stop rule against exhaustive KNN (Sec. III.B notes
    that the exploration may miss true neighbours): (recall@k, distance recall).

    recall@k: the share of the exact k neighbours, under (distance, index)
    order, that the walk returned.  Distance recall: the share of returned
    squared distances that are at most the exact k-th one.  Reported, not
    pinned: the paper's accuracy tables need its datasets.
    """
    ids, d2, _ = grid.query(queries, k, -1)
    e_ids, e_d2 = brute_force(points, queries, k)
    hit = sum(np.intersect1d(a[a >= 0], b[b >= 0]).size for a, b in zip(ids, e_ids))
    total = int((e_ids >= 0).sum())
    within = int((d2 <= e_d2[:, -1:]).sum())
    return hit / max(1, total), within / max(1, d2.size)
