"""Per-dimension cell widths, the paper's cell measurement and the certified
stop on the GPU, against the oracle (bit-exact).

* knn_measure_cells == oracle.measure_cells (split counts and widths), on
  uniform, clustered, tied, constant and one-dimensional data, from host and
  device memory;
* knn_build_grid with per-dimension widths, and with the measured widths and
  splits, queried under the paper's rule == the oracle's grid;
* KNN_QUERY_EXACT == the oracle's certified stop == exhaustive KNN, in the
  warp kernel, the cooperative kernel, the batched form and the no-alloc form.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2004_02290_gb300 import knn
from paper_2004_02290_gb300 import workloads as wl
from tests import refs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    return None if t is None else t.cpu().numpy() if isinstance(t, torch.Tensor) else t


def _same(got, exp, pred_too=True):
    ids, d2, pred = (_host(x) for x in got)
    e_ids, e_d2, e_pred = exp
    bad = np.nonzero((ids != e_ids).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:3]}: {ids[bad[0]]} vs {e_ids[bad[0]]}"
    assert np.array_equal(d2.view(np.uint32), e_d2.view(np.uint32))
    if pred_too and e_pred is not None:
        assert np.array_equal(pred.view(np.uint32), e_pred.view(np.uint32))


def _measure_inputs():
    rng = np.random.default_rng(12)
    cases = [wl.uniform(3000, 1, 3, seed=1)[0],
             np.concatenate([rng.normal(0.3, 0.01, (4000, 2)), rng.normal(0.8, 0.1, (500, 2))]),
             np.round(rng.normal(0.5, 0.2, (5000, 2)) * 40) / 40,
             np.concatenate([rng.random((2000, 1)), np.full((2000, 1), 0.25)], axis=1),
             rng.random((7, 4)),
             np.full((50, 2), 3.5),
             rng.random((1, 3))]
    cases.append(wl.make("large_cls", n=200_000, m=1, w=0.05).points)
    return [np.ascontiguousarray(c, np.float32) for c in cases]


@pytest.mark.parametrize("case", range(8))
def test_measure_cells_matches_oracle(case):
    x = _measure_inputs()[case]
    e_splits, e_widths = oracle.measure_cells(x)
    for src in (x, _dev(x)):
        splits, widths = knn.knn_measure_cells(src)
        assert splits.tolist() == e_splits.tolist()
        assert np.array_equal(widths.view(np.uint32), e_widths.view(np.uint32))


def test_measure_cells_rejects_non_finite():
    x = np.random.default_rng(0).random((100, 2)).astype(np.float32)
    x[7, 1] = np.inf
    with pytest.raises(knn.KnnError):
        knn.knn_measure_cells(_dev(x))


@pytest.mark.parametrize("table", [knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH])
@pytest.mark.parametrize("d,widths,k,mode", [
    (2, [0.02, 0.05], 5, knn.KNN_VOTE),
    (3, [0.1, 0.03, 0.07], 16, knn.KNN_MEAN),
    (4, [0.2, 0.1, 0.15, 0.12], 9, knn.KNN_MEDIAN),
    (6, [0.4, 0.3, 0.5, 0.35, 0.45, 0.3], 7, knn.KNN_VOTE),
])
def test_per_dimension_widths_match_oracle(d, widths, k, mode, table):
    x, lab, q = wl.uniform(5000, 300, d, seed=40 + d)
    if mode != knn.KNN_VOTE:
        lab = wl.regression_targets(x, seed=d)
    q = np.concatenate([q, np.full((2, d), -0.2, np.float32)]).astype(np.float32)
    w = np.array(widths, np.float32)
    idx = knn.knn_build_grid(_dev(x), _dev(lab), w, None, table)
    gw, gs = idx.grid()
    assert np.array_equal(gw, w) and (gs == 0).all()
    got = idx.query(_dev(q), k, mode, flags=knn.KNN_QUERY_CHECKED)
    _same(got, oracle.Grid(x, lab, w).query(q, k, mode))
    idx.free()


@pytest.mark.parametrize("seed,d,n", [(0, 2, 3000), (1, 3, 4000), (2, 2, 20000)])
def test_measured_grid_matches_oracle(seed, d, n):
    rng = np.random.default_rng(seed)
    x = np.round(rng.normal(0.5, 0.15, (n, d)) * 60) / 60  # ties: coarser measured grids
    x = x.astype(np.float32)
    lab = rng.integers(0, 5, size=n).astype(np.int32)
    q = rng.normal(0.5, 0.2, (200, d)).astype(np.float32)
    splits, widths = knn.knn_measure_cells(_dev(x))
    g = oracle.Grid(x, lab, widths, splits=splits)
    idx = knn.knn_build_grid(_dev(x), _dev(lab), widths, splits)
    inf = idx.info()
    assert [inf.extent[j] for j in range(d)] == splits.tolist()  # every split occupied
    for rule, flags in ((oracle.RULE_PAPER, 0), (oracle.RULE_EXACT, knn.KNN_QUERY_EXACT)):
        got = idx.query(_dev(q), 6, knn.KNN_VOTE, flags=flags | knn.KNN_QUERY_CHECKED)
        _same(got, g.query(q, 6, knn.KNN_VOTE, rule=rule))
    idx.free()


def _exhaustive(x, q, k):
    rows = [refs.knn_exhaustive(x, qi, k) for qi in q]
    return np.stack([r[0] for r in rows]), np.stack([r[1] for r in rows])


@pytest.mark.parametrize("table", [knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH])
@pytest.mark.parametrize("d,n,w,k", [(1, 3000, 0.002, 7), (2, 6000, 0.02, 16), (3, 8000, 0.05, 1),
                                     (4, 6000, 0.12, 40), (6, 3000, 0.35, 12), (8, 2000, 0.6, 5)])
def test_exact_flag_equals_exhaustive(d, n, w, k, table):
    x, lab, q = wl.uniform(n, 150, d, seed=70 + d)
    q = np.concatenate([q, np.full((2, d), -0.3), np.full((1, d), 1.6)]).astype(np.float32)
    idx = knn.knn_build(_dev(x), _dev(lab), w, table)
    got = idx.query(_dev(q), k, knn.KNN_VOTE, flags=knn.KNN_QUERY_EXACT | knn.KNN_QUERY_CHECKED)
    exp = oracle.Grid(x, lab, w).query(q, k, knn.KNN_VOTE, rule=oracle.RULE_EXACT)
    _same(got, exp)
    e_ids, e_d2 = _exhaustive(x, q, k)
    assert np.array_equal(_host(got[0]), e_ids)
    idx.free()


def test_exact_flag_on_clustered_data_and_lattice_ties():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0.3, 0.01, (5000, 3)), rng.random((500, 3))]).astype(np.float32)
    q = rng.random((300, 3)).astype(np.float32)
    idx = knn.knn_build(_dev(x), None, 0.02, knn.KNN_TABLE_HASH)
    got = idx.query(_dev(q), 10, knn.KNN_NONE, flags=knn.KNN_QUERY_EXACT | knn.KNN_QUERY_CHECKED)
    e_ids, e_d2 = _exhaustive(x, q, 10)
    assert np.array_equal(_host(got[0]), e_ids)
    assert np.array_equal(_host(got[1]).view(np.uint32), e_d2.view(np.uint32))
    idx.free()
    xl, labl, ql = wl.lattice(25, 2, 300, seed=4)
    idx = knn.knn_build(_dev(xl), _dev(labl), 1.0)
    got = idx.query(_dev(ql), 9, knn.KNN_VOTE, flags=knn.KNN_QUERY_EXACT | knn.KNN_QUERY_CHECKED)
    _same(got, oracle.Grid(xl, labl, 1.0).query(ql, 9, knn.KNN_VOTE, rule=oracle.RULE_EXACT))
    idx.free()


def test_exact_flag_in_batched_and_noalloc_forms():
    ps = wl.gen_batched(12, seed=21, n_lo=500, n_hi=20_000, dims=(2, 3, 4, 6), ks=(1, 5, 16, 40))
    for i, p in enumerate(ps):
        p.w = float(np.float32(0.04 * (1 + i % 3) * p.d / 3.0))
    b = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps],
                            [p.w for p in ps])
    ids, d2, pred = b.query([_dev(p.queries) for p in ps], [p.k for p in ps], [p.mode for p in ps],
                            flags=knn.KNN_QUERY_EXACT | knn.KNN_QUERY_CHECKED)
    for i, p in enumerate(ps):
        exp = oracle.Grid(p.points, p.labels, p.w).query(p.queries, p.k, p.mode,
                                                         rule=oracle.RULE_EXACT)
        _same((ids[i], d2[i], pred[i]), exp)
    b.free()
    p = ps[3]
    idx = knn.knn_build(_dev(p.points), _dev(p.labels), p.w)
    m = p.queries.shape[0]
    oi = torch.empty((m, p.k), dtype=torch.int32, device="cuda")
    od = torch.empty((m, p.k), dtype=torch.float32, device="cuda")
    op = torch.empty(m, dtype=torch.int32 if p.mode == knn.KNN_VOTE else torch.float32,
                     device="cuda")
    knn.knn_query_noalloc(idx, _dev(p.queries), p.k, p.mode, oi, od, op,
                          flags=knn.KNN_QUERY_EXACT | knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    _same((oi, od, op), oracle.Grid(p.points, p.labels, p.w).query(p.queries, p.k, p.mode,
                                                                   rule=oracle.RULE_EXACT))
    idx.free()


_FORCED = r"""
import numpy as np, torch, oracle
from paper_2004_02290_gb300 import knn, workloads as wl
def dev(a): return torch.from_numpy(np.ascontiguousarray(a)).cuda()
bad = 0
for d, n, w, k in [(2, 5000, 0.02, 10), (3, 6000, 0.05, 16), (4, 5000, 0.12, 40), (6, 2000, 0.35, 5)]:
    x, lab, q = wl.uniform(n, 120, d, seed=90 + d)
    q = np.concatenate([q, np.full((2, d), -0.4, np.float32)]).astype(np.float32)
    widths = np.float32(w) * (1.0 + 0.25 * np.arange(d, dtype=np.float32))
    e = oracle.Grid(x, lab, widths).query(q, k, 0, rule=oracle.RULE_EXACT)
    e2 = oracle.Grid(x, lab, widths).query(q, k, 0)
    for table in (knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH):
        idx = knn.knn_build_grid(dev(x), dev(lab), widths, None, table)
        for flags, exp in ((knn.KNN_QUERY_EXACT, e), (0, e2)):
            ids, d2, pred = idx.query(dev(q), k, 0, flags=flags | knn.KNN_QUERY_CHECKED)
            torch.cuda.synchronize()
            ok = (np.array_equal(ids.cpu().numpy(), exp[0])
                  and np.array_equal(d2.cpu().numpy().view(np.uint32), exp[1].view(np.uint32))
                  and np.array_equal(pred.cpu().numpy(), exp[2]))
            bad += not ok
        idx.free()
print("BAD", bad)
"""


def test_cooperative_kernel_exact_and_per_dimension_widths():
    """Every query forced through the cooperative kernel, exact and paper rule."""
    env = dict(os.environ, GHN_HEAVY_ROWS="2", GHN_HEAVY_CANDS="8", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", _FORCED], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "BAD 0" in r.stdout, r.stdout


@pytest.mark.parametrize("table", [knn.KNN_TABLE_DENSE, knn.KNN_TABLE_HASH])
@pytest.mark.parametrize("d,k,mode,rule", [
    (1, 64, knn.KNN_MEDIAN, oracle.RULE_PAPER),
    (5, 40, knn.KNN_MEAN, oracle.RULE_EXACT),
    (7, 33, knn.KNN_VOTE, oracle.RULE_PAPER),
    (8, 64, knn.KNN_MEDIAN, oracle.RULE_EXACT),
])
def test_wide_buffers_and_high_dimensions_per_dimension_widths(d, k, mode, rule, table):
    """Two-slot buffers (k > 32), d = 1, 5, 7, 8, every head, both rules."""
    x, lab, q = wl.uniform(3000, 120, d, seed=900 + d)
    if mode != knn.KNN_VOTE:
        lab = (np.round(wl.regression_targets(x, seed=d) * 8) / 8).astype(np.float32)
    w = (np.float32(0.08 + 0.07 * d) * (1.0 + 0.2 * np.arange(d))).astype(np.float32)
    q = np.concatenate([q, np.full((1, d), -0.25, np.float32)]).astype(np.float32)
    idx = knn.knn_build_grid(_dev(x), _dev(lab), w, None, table)
    flags = knn.KNN_QUERY_CHECKED | (knn.KNN_QUERY_EXACT if rule == oracle.RULE_EXACT else 0)
    got = idx.query(_dev(q), k, mode, flags=flags)
    _same(got, oracle.Grid(x, lab, w).query(q, k, mode, rule=rule))
    idx.free()


def test_measured_grid_one_dimension():
    rng = np.random.default_rng(44)
    x = np.round(rng.normal(0.5, 0.2, (4000, 1)) * 200).astype(np.float32) / np.float32(200)
    lab = rng.integers(0, 3, size=4000).astype(np.int32)
    q = rng.normal(0.5, 0.25, (300, 1)).astype(np.float32)
    splits, widths = knn.knn_measure_cells(_dev(x))
    e_splits, e_widths = oracle.measure_cells(x)
    assert splits.tolist() == e_splits.tolist() and np.array_equal(widths, e_widths)
    idx = knn.knn_build_grid(_dev(x), _dev(lab), widths, splits)
    got = idx.query(_dev(q), 9, knn.KNN_VOTE, flags=knn.KNN_QUERY_CHECKED)
    _same(got, oracle.Grid(x, lab, widths, splits=splits).query(q, 9, knn.KNN_VOTE))
    idx.free()


def test_exact_flag_with_locality_order_and_host_buffers():
    """KNN_QUERY_EXACT combined with KNN_QUERY_SORTED, and with host buffers."""
    x, lab, q = wl.uniform(8000, 500, 3, seed=77)
    q = np.concatenate([q, np.full((2, 3), 1.5, np.float32)]).astype(np.float32)
    exp = oracle.Grid(x, lab, 0.05).query(q, 12, knn.KNN_VOTE, rule=oracle.RULE_EXACT)
    idx = knn.knn_build(_dev(x), _dev(lab), 0.05)
    got = idx.query(_dev(q), 12, knn.KNN_VOTE,
                    flags=knn.KNN_QUERY_EXACT | knn.KNN_QUERY_SORTED | knn.KNN_QUERY_CHECKED)
    _same(got, exp)
    got_host = idx.query(q, 12, knn.KNN_VOTE, flags=knn.KNN_QUERY_EXACT | knn.KNN_QUERY_CHECKED)
    _same(got_host, exp)
    idx.free()
