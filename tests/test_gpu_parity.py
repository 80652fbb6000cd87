"""Parity of the CUDA path with the CPU oracle, through the C ABI (GPU needed).

Neighbour ids, squared distances and votes must be bit-exact; means must be
within 1e-6 relative (and are expected bit-exact: both sides sum the same
floats in double precision in the same order).  Small cases compare every
output; the full-size workloads compare a seeded sample of queries.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2004_02290_gb300 import knn
from paper_2004_02290_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MEAN_RTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_run(points, labels, queries, w, k, mode, table=knn.KNN_TABLE_AUTO, flags=0):
    idx = knn.knn_build(_dev(points), None if labels is None else _dev(labels), w, table)
    ids, d2, pred = idx.query(_dev(queries), k, mode, flags=flags | knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    info = idx.info()
    out = (ids.cpu().numpy(), d2.cpu().numpy(), None if pred is None else pred.cpu().numpy())
    idx.free()
    return out, info


def oracle_run(points, labels, queries, w, k, mode):
    g = oracle.Grid(points, labels, w)
    return g.query(queries, k, mode)


def assert_same(got, exp, mode):
    ids, d2, pred = got
    e_ids, e_d2, e_pred = exp
    assert ids.shape == e_ids.shape
    bad = np.nonzero((ids != e_ids).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:5]}: {ids[bad[0]]} vs {e_ids[bad[0]]}"
    assert np.array_equal(d2.view(np.uint32), e_d2.view(np.uint32))
    if mode == knn.KNN_VOTE:
        assert np.array_equal(pred, e_pred)
    elif mode == knn.KNN_MEAN:
        rel = np.abs(pred.astype(np.float64) - e_pred) / np.maximum(np.abs(e_pred), 1e-30)
        assert rel.max() <= MEAN_RTOL
        assert np.array_equal(pred.view(np.uint32), e_pred.view(np.uint32))
    elif mode == knn.KNN_MEDIAN:
        assert np.array_equal(pred.view(np.uint32), e_pred.view(np.uint32))


# ---- the tiny workload, every output ----

@pytest.mark.parametrize("flags", [0, knn.KNN_QUERY_SORTED])
@pytest.mark.parametrize("table", [knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH])
def test_tiny_workload(flags, table):
    w = wl.make("tiny")
    got, info = gpu_run(w.points, w.labels, w.queries, w.w, w.k, w.mode, table, flags)
    assert info.table == table
    assert_same(got, oracle_run(w.points, w.labels, w.queries, w.w, w.k, w.mode), w.mode)


def test_tiny_index_matches_algorithm1():
    """The built grid: the same occupied cells as the oracle, members in append order."""
    w = wl.make("tiny")
    for table in (knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH):
        idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w, table)
        info = idx.info()
        keys, starts, rows = idx.export()
        idx.free()
        g = oracle.Grid(w.points, w.labels, w.w)
        o, cmax = g.origin()
        assert np.array_equal(np.array(info.origin[:w.d], np.float32), o)
        assert list(info.extent[:w.d]) == (cmax + 1).tolist()
        coords, counts, members = g.cells()
        assert info.num_cells == g.num_cells
        ext = np.array(info.extent[:w.d], np.int64)
        strides = np.array([int(np.prod(ext[j + 1:])) for j in range(w.d)], np.int64)
        lin = (coords * strides).sum(axis=1)
        order = np.argsort(lin)
        assert np.array_equal(keys.astype(np.int64), lin[order])
        assert starts[-1] == w.n
        for c, e in enumerate(order):
            assert np.array_equal(rows[starts[c]:starts[c + 1]], members[e])


# ---- many shapes: d, k, tables, ties, outside queries ----

CASES = [
    # d, n, m, w, k, mode
    (1, 3000, 400, 0.002, 7, knn.KNN_VOTE),
    (2, 5000, 500, 0.02, 1, knn.KNN_VOTE),
    (2, 5000, 500, 0.02, 33, knn.KNN_VOTE),
    (3, 8000, 500, 0.05, 16, knn.KNN_MEAN),
    (4, 8000, 400, 0.12, 10, knn.KNN_VOTE),
    (4, 8000, 400, 0.12, 64, knn.KNN_MEAN),
    (5, 4000, 200, 0.3, 5, knn.KNN_VOTE),
    (6, 4000, 200, 0.35, 12, knn.KNN_MEAN),
    (7, 3000, 150, 0.45, 3, knn.KNN_VOTE),
    (8, 3000, 150, 0.5, 40, knn.KNN_VOTE),
]


@pytest.mark.parametrize("table", [knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH])
@pytest.mark.parametrize("d,n,m,w,k,mode", CASES)
def test_uniform_cases(d, n, m, w, k, mode, table):
    x, lab, q = wl.uniform(n, m, d, seed=1000 + 17 * d + k)
    if mode == knn.KNN_MEAN:
        lab = wl.regression_targets(x, seed=d)
    # queries also outside the box and on cell boundaries
    extra = np.stack([np.full(d, -0.3), np.full(d, 1.4), np.full(d, 0.5),
                      np.full(d, np.float32(w) * 3)]).astype(np.float32)
    q = np.concatenate([q, extra]).astype(np.float32)
    got, info = gpu_run(x, lab, q, w, k, mode, table)
    assert_same(got, oracle_run(x, lab, q, w, k, mode), mode)


@pytest.mark.parametrize("table", [knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH])
@pytest.mark.parametrize("d,n,m,w,k", [(2, 5000, 400, 0.02, 1), (2, 5000, 400, 0.02, 10),
                                       (3, 6000, 300, 0.06, 15), (4, 6000, 300, 0.12, 32),
                                       (4, 6000, 300, 0.12, 64), (6, 3000, 150, 0.35, 33)])
def test_median_cases(d, n, m, w, k, table):
    """Median head: bit-exact, with many equal outputs, signed zeros and even counts."""
    x, _, q = wl.uniform(n, m, d, seed=2000 + 13 * d + k)
    rng = np.random.default_rng(d + k)
    lab = (rng.integers(-3, 4, size=n) * 0.5).astype(np.float32)
    lab[rng.random(n) < 0.1] = np.float32(-0.0)
    q = np.concatenate([q, np.full((1, d), -0.3, np.float32)]).astype(np.float32)
    got, _ = gpu_run(x, lab, q, w, k, knn.KNN_MEDIAN, table)
    assert_same(got, oracle_run(x, lab, q, w, k, knn.KNN_MEDIAN), knn.KNN_MEDIAN)


def test_median_fewer_points_than_k():
    x = np.array([[0.1, 0.1], [0.2, 0.3], [0.9, 0.9]], np.float32)
    lab = np.array([3.0, -1.0, 2.0], np.float32)
    q = np.array([[0.0, 0.0], [1.0, 1.0]], np.float32)
    got, _ = gpu_run(x, lab, q, 0.25, 8, knn.KNN_MEDIAN)
    assert_same(got, oracle_run(x, lab, q, 0.25, 8, knn.KNN_MEDIAN), knn.KNN_MEDIAN)
    assert got[2][0] == np.float32(2.0)


def test_lattice_ties():
    """Integer lattice, w = 1: many exact distance ties, broken by the training index."""
    x, lab, q = wl.lattice(24, 2, 500, seed=3)
    for k in (1, 4, 9, 25, 64):
        for table in (knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH):
            got, _ = gpu_run(x, lab, q, 1.0, k, knn.KNN_VOTE, table)
            assert_same(got, oracle_run(x, lab, q, 1.0, k, knn.KNN_VOTE), knn.KNN_VOTE)


def test_lattice_3d_half_width():
    x, lab, q = wl.lattice(12, 3, 300, seed=4)
    got, _ = gpu_run(x, lab, q, 0.5, 8, knn.KNN_VOTE, knn.KNN_TABLE_HASH)
    assert_same(got, oracle_run(x, lab, q, 0.5, 8, knn.KNN_VOTE), knn.KNN_VOTE)


def test_single_cell_and_duplicates():
    """All points in one cell (w larger than the range), with exact duplicates."""
    x, lab, q = wl.uniform(2000, 300, 3, seed=7)
    x[500:900] = x[0]
    for table in (knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH):
        got, info = gpu_run(x, lab, q, 5.0, 20, knn.KNN_VOTE, table)
        assert info.num_cells == 1
        assert_same(got, oracle_run(x, lab, q, 5.0, 20, knn.KNN_VOTE), knn.KNN_VOTE)


@pytest.mark.parametrize("d", [2, 3, 5, 6])
@pytest.mark.parametrize("scale", [1e-20, 1e-21])
def test_subnormal_squared_distances(d, scale):
    """Coordinates near 1e-20: every squared difference is subnormal, so a
    flush to zero anywhere in the distance arithmetic (squares or sums)
    changes distance bits or the order of the neighbours."""
    x, lab, q = wl.uniform(3000, 200, d, seed=40 + d)
    x = (x * np.float32(scale)).astype(np.float32)
    q = (q * np.float32(scale)).astype(np.float32)
    w = float(np.float32(scale / 5))
    exp = oracle_run(x, lab, q, w, 8, knn.KNN_VOTE)
    assert (exp[1][exp[1] > 0] < np.float32(1.17549435e-38)).all()  # subnormal range
    for table in (knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH):
        got, _ = gpu_run(x, lab, q, w, 8, knn.KNN_VOTE, table)
        assert_same(got, exp, knn.KNN_VOTE)


@pytest.mark.parametrize("d,scale", [(2, 1e21), (4, 1.5e20), (5, 1e20)])
def test_overflowing_squared_distances(d, scale):
    """Coordinates near 1e20: most neighbours' squared distances overflow to
    +inf, so keys tie on the distance and the training index orders them,
    and the k-th distance is often infinite (no skipping)."""
    x, lab, q = wl.uniform(3000, 200, d, seed=50 + d)
    x = (x * np.float32(scale)).astype(np.float32)
    q = (q * np.float32(scale)).astype(np.float32)
    w = float(np.float32(scale / 8))
    exp = oracle_run(x, lab, q, w, 8, knn.KNN_VOTE)
    assert np.isinf(exp[1]).any() and np.isfinite(exp[1]).any()
    for table in (knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH):
        got, _ = gpu_run(x, lab, q, w, 8, knn.KNN_VOTE, table)
        assert_same(got, exp, knn.KNN_VOTE)


def test_k_larger_than_n():
    x, lab, q = wl.uniform(11, 40, 2, seed=8)
    for k in (11, 12, 64):
        got, _ = gpu_run(x, lab, q, 0.1, k, knn.KNN_VOTE)
        assert_same(got, oracle_run(x, lab, q, 0.1, k, knn.KNN_VOTE), knn.KNN_VOTE)
        assert (got[0][:, 11:] == -1).all() and np.isinf(got[1][:, 11:]).all()


def test_one_point():
    x = np.array([[0.25, -3.0]], np.float32)
    q = np.array([[0.0, 0.0], [1e6, -1e6], [0.25, -3.0]], np.float32)
    got, _ = gpu_run(x, np.array([5], np.int32), q, 0.7, 3, knn.KNN_VOTE)
    assert_same(got, oracle_run(x, np.array([5], np.int32), q, 0.7, 3, knn.KNN_VOTE), knn.KNN_VOTE)


def test_far_queries_clamped():
    x, lab, _ = wl.uniform(3000, 1, 2, seed=9)
    q = np.array([[1e30, 1e30], [-1e30, 0.5], [0.5, 3e9], [-7.0, -7.0]], np.float32)
    got, _ = gpu_run(x, lab, q, 0.05, 6, knn.KNN_VOTE)
    assert_same(got, oracle_run(x, lab, q, 0.05, 6, knn.KNN_VOTE), knn.KNN_VOTE)


def test_far_query_fine_grid():
    """Far queries on a fine grid: cell-unit gaps above 2^64 while distances stay finite."""
    x, lab, _ = wl.uniform(4000, 1, 2, seed=12, lo=0.0, hi=1e-4)
    q = np.array([[1e4, 1e4], [-1e4, 5e-5], [5e-5, 3e4], [2e-4, 2e-4]], np.float32)
    for k in (1, 7):
        got, _ = gpu_run(x, lab, q, 1e-6, k, knn.KNN_VOTE)
        assert_same(got, oracle_run(x, lab, q, 1e-6, k, knn.KNN_VOTE), knn.KNN_VOTE)


@pytest.mark.parametrize("flags", [0, knn.KNN_QUERY_SORTED])
@pytest.mark.parametrize("hi0,space", [(65535.5, 1 << 32), (65536.5, 65537 << 16)])
def test_cell_id_width_boundary(hi0, space, flags):
    """A box of exactly 2^32 cells (ids fill 32 bits: the build and the
    locality order sort 32-bit keys) and one just above it (64-bit keys)."""
    rng = np.random.default_rng(31)
    centres = np.array([[100.0, 100.0], [30000.0, 50000.0], [65000.0, 65000.0]])
    x = np.concatenate([c + 3.0 * rng.standard_normal((2000, 2)) for c in centres])
    x = np.clip(x, 0.0, 65535.5)
    x = np.concatenate([x, [[0.0, 0.0], [hi0, 65535.5]]]).astype(np.float32)
    lab = rng.integers(0, 4, len(x)).astype(np.int32)
    q = np.concatenate([c + 4.0 * rng.standard_normal((100, 2)) for c in centres]).astype(np.float32)
    got, info = gpu_run(x, lab, q, 1.0, 5, knn.KNN_VOTE, flags=flags)
    assert int(info.extent[0]) * int(info.extent[1]) == space
    assert info.table == knn.KNN_TABLE_HASH
    assert_same(got, oracle_run(x, lab, q, 1.0, 5, knn.KNN_VOTE), knn.KNN_VOTE)


@pytest.mark.parametrize("d,n", [(3, 4001), (5, 4003), (2, 3), (4, 4096)])
@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("where", ["device", "pinned"])
def test_point_alignment_and_tails(d, n, offset, where):
    """Points at a 16-byte boundary (the box and keys kernels load 4 points a
    thread, the last n mod 4 one by one) and one float past it (the scalar
    kernels), in device memory or in pinned host memory (copied first)."""
    x, lab, q = wl.uniform(n, 200, d, seed=40 + d)
    if where == "device":
        buf = torch.zeros(n * d + offset, dtype=torch.float32, device="cuda")
        buf[offset:] = torch.from_numpy(x).cuda().reshape(-1)
    else:
        buf = torch.zeros(n * d + offset, dtype=torch.float32).pin_memory()
        buf[offset:] = torch.from_numpy(x).reshape(-1)
    pts = buf[offset:].view(n, d)
    assert (pts.data_ptr() % 16 == 0) == (offset == 0)
    idx = knn.knn_build(pts, _dev(lab), 0.1)
    ids, d2, pred = idx.query(_dev(q), 4, knn.KNN_VOTE, flags=knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    info = idx.info()
    g = oracle.Grid(x, lab, 0.1)
    assert [float(info.origin[j]) for j in range(d)] == [float(v) for v in x.min(axis=0)]
    got = (ids.cpu().numpy(), d2.cpu().numpy(), pred.cpu().numpy())
    idx.free()
    assert_same(got, g.query(q, 4, knn.KNN_VOTE), knn.KNN_VOTE)


def test_clustered_heavy_cells():
    """Tight clusters: cells with thousands of points next to near-empty space."""
    w = wl.make("skewed_reg", n=200_000, m=3000, w=0.02)
    got, _ = gpu_run(w.points, w.labels, w.queries, w.w, w.k, w.mode)
    assert_same(got, oracle_run(w.points, w.labels, w.queries, w.w, w.k, w.mode), w.mode)


def test_large_cls_shape_small():
    w = wl.make("large_cls", n=100_000, m=5000, w=0.03)
    got, info = gpu_run(w.points, w.labels, w.queries, w.w, w.k, w.mode, knn.KNN_TABLE_HASH,
                        knn.KNN_QUERY_SORTED)
    assert info.table == knn.KNN_TABLE_HASH
    assert_same(got, oracle_run(w.points, w.labels, w.queries, w.w, w.k, w.mode), w.mode)


# ---- counters of the method's work (exhaustive walk) ----

@pytest.mark.parametrize("table", [knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH])
def test_stats_match_oracle(table):
    w = wl.make("tiny")
    idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w, table)
    ids, d2, st = idx.query_stats(_dev(w.queries), w.k)
    ids_q, d2_q, _ = idx.query(_dev(w.queries), w.k)
    torch.cuda.synchronize()
    g = oracle.Grid(w.points, w.labels, w.w)
    e_ids, e_d2, _, e_st = g.query(w.queries, w.k, -1, stats=True)
    assert np.array_equal(st.cpu().numpy(), e_st)
    assert np.array_equal(ids.cpu().numpy(), e_ids)
    # the skipping walk gives the same result as the exhaustive one
    assert np.array_equal(ids_q.cpu().numpy(), e_ids)
    assert np.array_equal(d2_q.cpu().numpy().view(np.uint32), e_d2.view(np.uint32))
    idx.free()


# ---- host buffers, empty and invalid input, determinism ----

def test_host_buffers_match_device_buffers():
    w = wl.make("tiny")
    idx = knn.knn_build(w.points, w.labels, w.w)  # numpy: host pointers
    ids, d2, pred = idx.query(w.queries, w.k, knn.KNN_VOTE)
    assert isinstance(ids, np.ndarray)
    assert_same((ids, d2, pred), oracle_run(w.points, w.labels, w.queries, w.w, w.k, w.mode),
                knn.KNN_VOTE)
    idx.free()


@pytest.mark.parametrize("mode", [knn.KNN_VOTE, knn.KNN_MEAN])
def test_pinned_host_buffers(mode):
    """Pinned host inputs and outputs: the labels are copied into the index on a
    side stream during the build, and the kernels write ids, distances and
    predictions straight into the pinned outputs.  Pageable outputs (numpy)
    and device outputs give the same bytes."""
    w = wl.make("large_cls", n=60_000, m=4_000, w=0.04)
    lab = w.labels if mode == knn.KNN_VOTE else w.labels.astype(np.float32) * 0.5
    pts_h = torch.from_numpy(w.points).pin_memory()
    lab_h = torch.from_numpy(lab).pin_memory()
    q_h = torch.from_numpy(w.queries).pin_memory()
    idx = knn.knn_build(pts_h, lab_h, w.w)
    ids = torch.full((w.m, w.k), -7, dtype=torch.int32).pin_memory()
    d2 = torch.full((w.m, w.k), -7.0, dtype=torch.float32).pin_memory()
    pred = torch.full((w.m,), -7, dtype=torch.int32 if mode == knn.KNN_VOTE else torch.float32)
    pred = pred.pin_memory()
    knn.knn_query(idx, q_h, w.k, mode, flags=knn.KNN_QUERY_CHECKED, ids=ids, dist2=d2, pred=pred)
    got = (ids.numpy(), d2.numpy(), pred.numpy())  # filled when the call returns
    assert_same(got, oracle_run(w.points, lab, w.queries, w.w, w.k, mode), mode)
    pg = idx.query(w.queries, w.k, mode)  # pageable host outputs (staged copies)
    dv = idx.query(_dev(w.queries), w.k, mode)  # device outputs
    torch.cuda.synchronize()
    for a, b_, c in zip(got, pg, dv):
        assert np.array_equal(a.view(np.uint32), np.asarray(b_).view(np.uint32))
        assert np.array_equal(a.view(np.uint32), c.cpu().numpy().view(np.uint32))
    idx.free()


def test_phase_timing_reads_calls_oldest_first():
    w = wl.make("tiny")
    knn.knn_timing_enable(True)
    try:
        idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w)
        idx.query(_dev(w.queries), w.k, knn.KNN_VOTE)
        idx.query(_dev(w.queries), w.k, knn.KNN_VOTE, flags=knn.KNN_QUERY_SORTED)
        build = knn.knn_timing_read()
        q1 = knn.knn_timing_read()
        q2 = knn.knn_timing_read()
        # tiny is a small dense index: one launch builds it ("small")
        assert [n for n, _ in build] == ["stage", "box", "small", "gather"]
        # search: the warp or slot kernel; coop: the cooperative kernel
        assert [n for n, _ in q1] == [n for n, _ in q2] == ["stage", "order", "search", "coop",
                                                            "copy"]
        assert all(t >= 0.0 for _, t in build + q1 + q2)
        assert knn.knn_timing_read() == []
        # the thread keeps its last 32 calls: the oldest unread ones are dropped
        for _ in range(40):
            idx.query(_dev(w.queries[:10]), 1)
        got = 0
        while knn.knn_timing_read():
            got += 1
        assert got == 32
        idx.free()
    finally:
        knn.knn_timing_enable(False)


def test_empty_query_batch():
    w = wl.make("tiny")
    idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w)
    ids, d2, pred = idx.query(_dev(np.zeros((0, 2), np.float32)), 5, knn.KNN_VOTE,
                              flags=knn.KNN_QUERY_CHECKED)
    assert ids.shape == (0, 5)
    idx.free()


def test_non_finite_query_is_reported():
    w = wl.make("tiny")
    idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w)
    q = w.queries[:10].copy()
    q[3, 1] = np.nan
    with pytest.raises(knn.KnnError) as e:
        idx.query(_dev(q), 5, knn.KNN_VOTE, flags=knn.KNN_QUERY_CHECKED)
    assert e.value.code == knn.KNN_EINVAL
    ids, d2, _ = idx.query(_dev(q), 5, knn.KNN_VOTE)
    torch.cuda.synchronize()
    ids = ids.cpu().numpy()
    assert (ids[3] == -1).all() and (ids[[0, 1, 2, 4]] >= 0).all()
    idx.free()


def test_non_finite_point_is_rejected():
    x, lab, _ = wl.uniform(100, 1, 2, seed=1)
    x[7, 0] = np.inf
    with pytest.raises(knn.KnnError) as e:
        knn.knn_build(_dev(x), _dev(lab), 0.1)
    assert e.value.code == knn.KNN_EINVAL


def test_grid_too_fine_is_rejected():
    x, lab, _ = wl.uniform(100, 1, 3, seed=1)
    with pytest.raises(knn.KnnError) as e:
        knn.knn_build(_dev(x), _dev(lab), 1e-12)
    assert e.value.code == knn.KNN_EINVAL
    with pytest.raises(knn.KnnError) as e:
        knn.knn_build(_dev(x), _dev(lab), 1e-4, knn.KNN_TABLE_DENSE)
    assert e.value.code == knn.KNN_EINVAL


def test_prediction_without_labels_is_rejected():
    x, _, q = wl.uniform(100, 5, 2, seed=1)
    idx = knn.knn_build(_dev(x), None, 0.1)
    with pytest.raises(knn.KnnError):
        idx.query(_dev(q), 3, knn.KNN_VOTE)
    ids, _, _ = idx.query(_dev(q), 3, knn.KNN_NONE, flags=knn.KNN_QUERY_CHECKED)
    assert ids.shape == (5, 3)
    idx.free()


def test_deterministic_bytes():
    w = wl.make("large_cls", n=50_000, m=4000, w=0.03)
    a, _ = gpu_run(w.points, w.labels, w.queries, w.w, w.k, w.mode, knn.KNN_TABLE_HASH)
    b, _ = gpu_run(w.points, w.labels, w.queries, w.w, w.k, w.mode, knn.KNN_TABLE_HASH)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _child(code, env):
    e = dict(os.environ, **env)
    return subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=e, capture_output=True,
                          text=True, timeout=300)


@pytest.mark.parametrize("n,ats", [(1000, ("1", "3", "6")),          # one-launch small build
                                   (40000, ("1", "3", "9", "12"))])  # multi-kernel build
def test_injected_allocation_failure(n, ats):
    code = (
        "import numpy as np, torch\n"
        "from paper_2004_02290_gb300 import knn, workloads as wl\n"
        f"x, lab, q = wl.uniform({n}, 10, 2, seed=1)\n"
        "try:\n"
        "    knn.knn_build(torch.from_numpy(x).cuda(), torch.from_numpy(lab).cuda(), 0.05)\n"
        "    print('NOFAIL')\n"
        "except knn.KnnError as e:\n"
        "    print('CODE', e.code)\n"
        "idx = knn.knn_build(torch.from_numpy(x).cuda(), torch.from_numpy(lab).cuda(), 0.05)\n"
        "ids, _, _ = idx.query(torch.from_numpy(q).cuda(), 3, flags=knn.KNN_QUERY_CHECKED)\n"
        "print('AFTER', int(ids.min()))\n")
    for at in ats:
        r = _child(code, {"GHN_FAIL_ALLOC_AT": at})
        assert r.returncode == 0, r.stderr
        assert "CODE 2" in r.stdout, (at, r.stdout)
        # the next build and query work: every id found is a training index
        assert int(r.stdout.split("AFTER")[1].split()[0]) >= 0, (at, r.stdout)


def test_layer_cap_reports_limit():
    code = (
        "import numpy as np, torch\n"
        "from paper_2004_02290_gb300 import knn, workloads as wl\n"
        "x, lab, q = wl.uniform(5000, 200, 2, seed=2)\n"
        "idx = knn.knn_build(torch.from_numpy(x).cuda(), torch.from_numpy(lab).cuda(), 0.01)\n"
        "try:\n"
        "    idx.query(torch.from_numpy(q).cuda(), 8, flags=knn.KNN_QUERY_CHECKED)\n"
        "    print('NOFAIL')\n"
        "except knn.KnnError as e:\n"
        "    print('CODE', e.code)\n"
        "ids, _, _ = idx.query(torch.from_numpy(q).cuda(), 8)\n"
        "torch.cuda.synchronize()\n"
        "print('NEG', int((ids.cpu().numpy() == -1).all(axis=1).sum()))\n")
    r = _child(code, {"GHN_MAX_LAYERS": "1"})
    assert r.returncode == 0, r.stderr
    assert "CODE 4" in r.stdout, r.stdout
    neg = int(r.stdout.split("NEG")[1].split()[0])
    assert neg > 0


def test_default_work_bound_trips_on_a_grid_far_finer_than_k_th_distance():
    """2,000 points in the unit square on cells of 2e-6: the 8th neighbour is
    about 0.036 away, some 18,000 layers out.  The default bound (2^22 rows
    enumerated; in 2-D, layer L has 2L + 1 rows) ends each walk after about
    2,048 layers (0.004 away, where a query expects 0.1 points): KNN_ELIMIT
    under KNN_QUERY_CHECKED, -1 / +inf rows, and the call returns within
    seconds."""
    import time

    rng = np.random.default_rng(77)
    x = rng.random((2000, 2)).astype(np.float32)
    lab = rng.integers(0, 3, 2000).astype(np.int32)
    q = rng.random((16, 2)).astype(np.float32)
    idx = knn.knn_build(_dev(x), _dev(lab), 2e-6)
    t0 = time.perf_counter()
    with pytest.raises(knn.KnnError) as e:
        idx.query(_dev(q), 8, knn.KNN_VOTE, flags=knn.KNN_QUERY_CHECKED)
    assert e.value.code == knn.KNN_ELIMIT
    assert time.perf_counter() - t0 < 30.0
    ids, d2, _ = idx.query(_dev(q), 8, knn.KNN_VOTE)
    torch.cuda.synchronize()
    assert (ids.cpu().numpy() == -1).all() and np.isinf(d2.cpu().numpy()).all()
    idx.free()


def test_work_bound_override():
    """GHN_MAX_ROWS replaces the default bound: 3 rows stop every walk that
    needs layer 1 (3 rows in 2-D after the central row)."""
    code = (
        "import numpy as np, torch\n"
        "from paper_2004_02290_gb300 import knn, workloads as wl\n"
        "x, lab, q = wl.uniform(5000, 200, 2, seed=2)\n"
        "idx = knn.knn_build(torch.from_numpy(x).cuda(), torch.from_numpy(lab).cuda(), 0.01)\n"
        "try:\n"
        "    idx.query(torch.from_numpy(q).cuda(), 8, flags=knn.KNN_QUERY_CHECKED)\n"
        "    print('NOFAIL')\n"
        "except knn.KnnError as e:\n"
        "    print('CODE', e.code)\n")
    r = _child(code, {"GHN_MAX_ROWS": "3"})
    assert r.returncode == 0, r.stderr
    assert "CODE 4" in r.stdout, r.stdout
    r = _child(code, {"GHN_MAX_ROWS": "0"})  # no bound
    assert r.returncode == 0, r.stderr
    assert "NOFAIL" in r.stdout, r.stdout


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second GPU")
def test_buffers_of_another_gpu_are_refused():
    x, lab, q = wl.uniform(1000, 8, 2, seed=3)
    idx = knn.knn_build(_dev(x), _dev(lab), 0.05)
    q1 = torch.from_numpy(q).to("cuda:1")
    with pytest.raises(knn.KnnError) as e:
        idx.query(q1, 3, knn.KNN_VOTE, flags=knn.KNN_QUERY_CHECKED)
    assert e.value.code == knn.KNN_EINVAL
    idx.free()


_BUILD_CASES = r"""
import sys, numpy as np, torch
from paper_2004_02290_gb300 import knn, workloads as wl
def dev(a): return torch.from_numpy(np.ascontiguousarray(a)).cuda()
out = {}
cases = [(1, 3000, 0.002), (2, 10000, 0.018), (3, 16384, 0.09), (4, 5000, 0.25), (6, 2000, 0.6),
         (8, 1500, 0.9), (2, 1, 0.5), (3, 777, 0.05)]
for ci, (d, n, w) in enumerate(cases):
    x, lab, q = wl.uniform(n, 200, d, seed=70 + ci)
    if ci == 1:
        x, lab, q = wl.make("tiny").points, wl.make("tiny").labels, wl.make("tiny").queries
    idx = knn.knn_build(dev(x), dev(lab), w, knn.KNN_TABLE_DENSE)
    inf = idx.info()
    u = int(inf.num_cells)
    keys = np.zeros(u, np.uint64); starts = np.zeros(u + 1, np.uint32); rows = np.zeros(len(x), np.int32)
    lib = knn.library()
    assert lib.knn_index_export(idx.handle, keys.ctypes.data, starts.ctypes.data, rows.ctypes.data) == 0
    ids, d2, pred = idx.query(dev(q), 7, knn.KNN_VOTE, flags=knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    out[f"{ci}_k"] = keys; out[f"{ci}_s"] = starts; out[f"{ci}_r"] = rows
    out[f"{ci}_i"] = ids.cpu().numpy(); out[f"{ci}_d"] = d2.cpu().numpy(); out[f"{ci}_p"] = pred.cpu().numpy()
    out[f"{ci}_u"] = np.array([u, inf.table], np.int64)
    idx.free()
np.savez(sys.argv[1], **out)
"""


def test_small_build_equals_the_multi_kernel_build(tmp_path):
    """The one-launch build of small dense indexes (n <= 16384, at most 32767
    cells) and the multi-kernel build (GHN_SMALL_BUILD=0) give the same cell
    list, row order and query outputs (one point, n = 16384, d = 1..8)."""
    res = {}
    for name, env in (("small", {}), ("multi", {"GHN_SMALL_BUILD": "0"})):
        path = str(tmp_path / f"{name}.npz")
        r = subprocess.run([sys.executable, "-c", _BUILD_CASES, path], cwd=ROOT,
                           env=dict(os.environ, **env), capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr[-3000:]
        res[name] = np.load(path)
    a, b = res["small"], res["multi"]
    assert sorted(a.files) == sorted(b.files)
    for f in a.files:
        assert np.array_equal(a[f].view(np.uint8), b[f].view(np.uint8)), f


# ---- full-size workloads, in the benchmark's launch configuration, sampled ----

def _sampled_full(name, sample, flags):
    w = wl.make(name)
    idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w, w.table)
    ids, d2, pred = idx.query(_dev(w.queries), w.k, w.mode, flags=flags | knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    rng = np.random.default_rng(123)
    pick = np.sort(rng.choice(w.m, size=sample, replace=False))
    g = oracle.Grid(w.points, w.labels, w.w)
    rule = oracle.RULE_EXACT if flags & knn.KNN_QUERY_EXACT else oracle.RULE_PAPER
    exp = g.query(w.queries[pick], w.k, w.mode, rule=rule)
    got = (ids.cpu().numpy()[pick], d2.cpu().numpy()[pick], pred.cpu().numpy()[pick])
    assert_same(got, exp, w.mode)
    # properties that hold for every row: sorted, distinct, in range
    allids = ids.cpu().numpy()
    alld = d2.cpu().numpy()
    assert (allids >= 0).all() and (allids < w.n).all()
    assert (np.diff(alld, axis=1) >= 0).all()
    s = np.sort(allids, axis=1)
    assert (np.diff(s, axis=1) > 0).all()
    idx.free()


def test_full_large_cls_sampled():
    import bench

    _sampled_full("large_cls", 3000, bench.query_flags(knn, "large_cls"))


def test_full_large_cls_sampled_sorted():
    _sampled_full("large_cls", 1000, knn.KNN_QUERY_SORTED)


def test_full_skewed_reg_sampled():
    import bench

    _sampled_full("skewed_reg", 1500, bench.query_flags(knn, "skewed_reg"))


def test_full_skewed_reg_sampled_input_order():
    _sampled_full("skewed_reg", 800, 0)


def test_full_large_cls_sampled_certified_stop():
    _sampled_full("large_cls", 1500, knn.KNN_QUERY_EXACT)


def test_full_skewed_reg_sampled_certified_stop():
    _sampled_full("skewed_reg", 800, knn.KNN_QUERY_EXACT)


_FORCED_DEFERRAL = r"""
import numpy as np, torch, oracle
from paper_2004_02290_gb300 import knn, workloads as wl
def dev(a): return torch.from_numpy(np.ascontiguousarray(a)).cuda()
cases = []
for d, n, m, w, k in [(2, 5000, 300, 0.02, 10), (3, 8000, 300, 0.05, 16), (4, 8000, 200, 0.12, 40),
                      (1, 3000, 200, 0.002, 7), (6, 3000, 100, 0.35, 5)]:
    x, lab, q = wl.uniform(n, m, d, seed=500 + d)
    q = np.concatenate([q, np.full((2, d), -0.4, np.float32), np.full((1, d), 1.3, np.float32)])
    cases.append((x, lab, q.astype(np.float32), w, k))
x, lab, q = wl.lattice(20, 2, 200, seed=6)
cases.append((x, lab, q, 1.0, 9))
cw = wl.make("skewed_reg", n=100_000, m=1000, w=0.02)
cases.append((cw.points, cw.labels, cw.queries, cw.w, 16))
bad = 0
for x, lab, q, w, k in cases:
    g = oracle.Grid(x, lab, w)
    modes = [knn.KNN_VOTE] if lab.dtype == np.int32 else [knn.KNN_MEAN, knn.KNN_MEDIAN]
    for mode in modes:
        e_ids, e_d2, e_pred = g.query(q, k, mode)
        for table in (knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH):
            idx = knn.knn_build(dev(x), dev(lab), w, table)
            ids, d2, pred = idx.query(dev(q), k, mode,
                                      flags=knn.KNN_QUERY_CHECKED | knn.KNN_QUERY_SORTED)
            torch.cuda.synchronize()
            ok = (np.array_equal(ids.cpu().numpy(), e_ids)
                  and np.array_equal(d2.cpu().numpy().view(np.uint32), e_d2.view(np.uint32))
                  and np.array_equal(pred.cpu().numpy().view(np.uint32), e_pred.view(np.uint32)))
            bad += not ok
            idx.free()
print("BAD", bad)
"""


def test_cooperative_kernel_parity():
    """Every query forced through the cooperative (block-per-query) kernel."""
    r = _child(_FORCED_DEFERRAL, {"GHN_HEAVY_ROWS": "2", "GHN_HEAVY_CANDS": "8"})
    assert r.returncode == 0, r.stderr[-3000:]
    assert "BAD 0" in r.stdout, r.stdout
