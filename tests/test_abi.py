"""The C ABI library loads, exports what include/ghn_knn.h declares, and rejects
bad arguments on the host before touching a GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2004_02290_gb300 import knn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("ghn_knn.h", "ghn_serve.h")]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return knn.library()


def _declared():
    text = ""
    for h in HEADERS:
        with open(h) as f:
            text += f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(knn_[a-z_]+)\s*\(", text)))


def test_header_declares_build_query_and_free():
    names = _declared()
    for required in ("knn_build", "knn_query", "knn_free"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} is declared in ghn_knn.h but not exported"
    assert sorted(_declared()) == sorted(knn.EXPORTED)


def test_abi_version(lib):
    assert lib.knn_abi_version() == 1


def _build_status(lib, points, labels, n, d, w, table=0):
    h = ctypes.c_void_p()
    rc = lib.knn_build(points, labels, n, d, ctypes.c_float(w), table, None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("n,d,w,table,why", [
    (0, 2, 1.0, 0, "n = 0"),
    (-5, 2, 1.0, 0, "n < 0"),
    (1 << 31, 2, 1.0, 0, "n"),
    (10, 0, 1.0, 0, "d = 0"),
    (10, 9, 1.0, 0, "d = 9"),
    (10, 2, 0.0, 0, "cell width"),
    (10, 2, -1.0, 0, "cell width"),
    (10, 2, float("inf"), 0, "cell width"),
    (10, 2, float("nan"), 0, "cell width"),
    (10, 2, 1.0, 3, "table"),
])
def test_build_rejects_bad_arguments(lib, n, d, w, table, why):
    buf = (ctypes.c_float * 64)()
    rc, h = _build_status(lib, ctypes.addressof(buf), None, n, d, w, table)
    assert rc == knn.KNN_EINVAL
    assert not h.value
    assert lib.knn_last_error()


def test_build_rejects_null_points(lib):
    rc, _ = _build_status(lib, None, None, 10, 2, 1.0)
    assert rc == knn.KNN_EINVAL
    assert b"points" in lib.knn_last_error()


def test_build_rejects_null_out(lib):
    buf = (ctypes.c_float * 8)()
    rc = lib.knn_build(ctypes.addressof(buf), None, 4, 2, ctypes.c_float(1.0), 0, None, None)
    assert rc == knn.KNN_EINVAL


def test_query_rejects_null_index(lib):
    ids = (ctypes.c_int32 * 8)()
    q = (ctypes.c_float * 8)()
    rc = lib.knn_query(None, ctypes.addressof(q), 1, 3, -1, ctypes.addressof(ids), None, None, 0,
                       None)
    assert rc == knn.KNN_EINVAL
    assert b"index" in lib.knn_last_error()


def test_free_null_is_a_noop(lib):
    lib.knn_free(None)


def test_python_binding_has_the_abi_names():
    for name in ("knn_build", "knn_query", "knn_query_stats", "knn_free", "knn_last_error"):
        assert callable(getattr(knn, name))


def test_binding_refuses_missing_library(tmp_path):
    # the binding never falls back to another implementation
    saved = knn._lib
    try:
        knn._lib = None
        with pytest.raises(RuntimeError):
            knn.library(str(tmp_path / "missing.so"))
    finally:
        knn._lib = saved


def test_batch_build_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 1)(10)
    d = (ctypes.c_int32 * 1)(2)
    w = (ctypes.c_float * 1)(1.0)
    pts = (ctypes.c_void_p * 1)(None)
    assert lib.knn_batch_build(0, pts, None, n, d, w, None, None, ctypes.byref(h)) == knn.KNN_EINVAL
    bad_d = (ctypes.c_int32 * 1)(9)
    assert lib.knn_batch_build(1, pts, None, n, bad_d, w, None, None,
                               ctypes.byref(h)) == knn.KNN_EINVAL
    bad_w = (ctypes.c_float * 1)(-1.0)
    assert lib.knn_batch_build(1, pts, None, n, d, bad_w, None, None,
                               ctypes.byref(h)) == knn.KNN_EINVAL
    assert not h.value
    lib.knn_batch_free(None)
    lib.knn_plan_free(None)


def test_server_rejects_bad_arguments_on_the_host(lib):
    """Checks that need no GPU: NULL pointers, bad configuration fields, bad requests."""
    h = ctypes.c_void_p()
    assert lib.knn_server_create(None, None) == knn.KNN_EINVAL
    bad = knn.knn_server_config(0, 0, 0, 0, 0, 0, 7)  # reserved must be 0
    assert lib.knn_server_create(ctypes.byref(bad), ctypes.byref(h)) == knn.KNN_EINVAL
    assert not h.value
    bad = knn.knn_server_config(0, -5, 0, 0, 0, 0, 0)
    assert lib.knn_server_create(ctypes.byref(bad), ctypes.byref(h)) == knn.KNN_EINVAL
    t = ctypes.c_int64()
    assert lib.knn_server_submit(None, 1, None, 0, 5, -1, None, None, None, 0,
                                 ctypes.byref(t)) == knn.KNN_EINVAL
    assert lib.knn_server_wait(None, 1, 0, None) == knn.KNN_EINVAL
    assert lib.knn_server_drop(None, 1, ctypes.byref(t)) == knn.KNN_EINVAL
    assert lib.knn_server_stats(None, None) == knn.KNN_EINVAL
    lib.knn_server_destroy(None)


def test_server_build_bound_grows_with_n(lib):
    a = lib.knn_server_build_bytes(1000, 3, 1)
    b = lib.knn_server_build_bytes(2000, 3, 1)
    assert 0 < a < b
    assert lib.knn_server_build_bytes(1000, 6, 1) > a  # wider rows
    assert lib.knn_server_build_bytes(0, 3, 1) == 0
    assert lib.knn_server_build_bytes(10, 9, 1) == 0


def test_server_clock_is_monotonic_ns(lib):
    import time

    a = time.monotonic_ns()
    c = lib.knn_server_clock_ns()
    b = time.monotonic_ns()
    assert a <= c <= b
