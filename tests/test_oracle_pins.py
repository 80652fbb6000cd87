"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: the expected values are the
paper's closed forms (Eq. 2, Eq. 3), its worked example (Sec. III.B), hand
derivations stored under tests/golden/, an exhaustive numpy KNN, and the set
form of the stop rule restated in numpy (tests/refs.py).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2004_02290_gb300 import workloads as wl
from tests import refs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---- Eq. 2 and Eq. 3: the number of cells per layer ----

@pytest.mark.parametrize("d", range(1, 9))
def test_eq2_cells_on_layer(d):
    """Eq. 2 (Sec. III.C, App. A): layer l holds (2l+1)^d - (2l-1)^d cells."""
    max_l = {1: 6, 2: 6, 3: 5, 4: 4, 5: 3, 6: 2, 7: 2, 8: 2}[d]
    assert oracle.shell_count(d, 0) == 1  # layer 0 is the central cell alone
    for L in range(1, max_l + 1):
        assert oracle.shell_count(d, L) == (2 * L + 1) ** d - (2 * L - 1) ** d


@pytest.mark.parametrize("d", range(1, 9))
def test_eq3_cumulative_cells(d):
    """Eq. 3 (App. B): layers 1..l hold (2l+1)^d - 1 cells (central cell excluded)."""
    max_l = {1: 6, 2: 6, 3: 5, 4: 4, 5: 3, 6: 2, 7: 2, 8: 2}[d]
    total = 0
    for L in range(1, max_l + 1):
        total += oracle.shell_count(d, L)
        assert total == (2 * L + 1) ** d - 1


def test_best_case_layer1_count():
    """Sec. III.C best case: stopping after layer 1 visits 3^d - 1 cells around the centre."""
    for d in range(1, 9):
        assert oracle.shell_count(d, 1) == 3 ** d - 1


# ---- Eq. 1: cell ids, hand-derived ----

@pytest.mark.parametrize("case", _golden("cell_keys.json")["cases"], ids=lambda c: c["name"])
def test_eq1_cell_ids(case):
    g = oracle.Grid(np.array(case["train"], np.float32), None, case["w"])
    got = g.cells_of(np.array(case["probe"], np.float32), as_query=case["as_query"])
    assert got.tolist() == case["cells"], case["why"]


def test_origin_and_box():
    x, lab, _ = wl.uniform(500, 1, 3, seed=5, lo=-2.0, hi=3.0)
    g = oracle.Grid(x, lab, 0.37)
    o, cmax = g.origin()
    assert np.array_equal(o, x.min(axis=0))
    coords, _, _ = g.cells()
    assert np.array_equal(cmax, coords.max(axis=0))
    assert coords.min() == 0


# ---- Algorithm 1: cell sampling invariants ----

@pytest.mark.parametrize("d,n,w", [(1, 300, 0.05), (2, 2000, 0.03), (3, 3000, 0.11),
                                   (5, 800, 0.4), (8, 500, 0.7)])
def test_alg1_invariants(d, n, w):
    x, lab, _ = wl.uniform(n, 1, d, seed=d * 7 + 1)
    g = oracle.Grid(x, lab, w)
    coords, counts, members = g.cells()
    u = g.num_cells
    # every point lands in exactly one cell, and cell sizes sum to n
    allm = np.concatenate(members)
    assert counts.sum() == n
    assert np.array_equal(np.sort(allm), np.arange(n))
    # the number of cells never exceeds n; no empty cell is stored (Sec. III.A, III.C)
    assert 1 <= u <= n
    assert (counts >= 1).all()
    # distinct cell ids
    assert len({tuple(c) for c in coords.tolist()}) == u
    # each member's cell id is its cell's id; members keep input order (append)
    pc = g.cells_of(x)
    for e in range(u):
        assert (pc[members[e]] == coords[e]).all()
        assert (np.diff(members[e]) > 0).all()


def test_alg1_duplicates_share_a_cell():
    x = np.array([[0.1, 0.1]] * 5 + [[0.9, 0.9]] * 3, np.float32)
    g = oracle.Grid(x, np.zeros(8, np.int32), 0.2)
    _, counts, members = g.cells()
    assert sorted(counts.tolist()) == [3, 5]
    assert sorted(m.tolist() for m in members) == [[0, 1, 2, 3, 4], [5, 6, 7]]


# ---- Sec. III.B: the worked example ----

def test_worked_example_sec3b():
    ex = _golden("worked_example_2d.json")
    pts = np.array(ex["points"], np.float32)
    g = oracle.Grid(pts, np.zeros(len(pts), np.int32), ex["w"])
    q = np.array(ex["query"], np.float32)
    assert g.cells_of(q[None], as_query=True)[0].tolist() == ex["central_cell"]
    c0 = np.array(ex["central_cell"])
    cheb = np.abs(g.cells_of(pts) - c0).max(axis=1)
    assert cheb.tolist() == ex["layer_of_point"]
    for L, cnt in ex["cells_on_layer"].items():
        assert oracle.shell_count(2, int(L)) == cnt
    ids, d2, _, st = g.query_one(q, ex["k"])
    assert ids.tolist() == ex["expected_ids"]
    assert st.tolist() == [ex["expected_layers_visited"], ex["expected_occupied_cells_looked_up"],
                           ex["expected_points_examined"]]
    # the distances are the float32 squared distances of those points
    assert np.array_equal(d2, refs.sqdist_f32(pts, q)[ids])
    # the narrative: after layer 0 the buffer is short, layer 1 updates, layer 2 does not
    ids0, _, _ = refs.set_form(pts, g.cells_of(pts), q, c0, g.origin()[1], ex["k"])[:3]
    assert ids0.tolist() == ex["expected_ids"]


# ---- original KNN, and the exhaustive special cases ----

@pytest.mark.parametrize("d", [1, 2, 3, 4, 6, 8])
def test_brute_force_matches_numpy(d):
    x, _, q = wl.uniform(300, 20, d, seed=100 + d)
    for k in (1, 5, 300, 305):
        ids, d2 = oracle.brute_force(x, q, k)
        for i in range(q.shape[0]):
            e_ids, e_d2 = refs.knn_exhaustive(x, q[i], k)
            assert np.array_equal(ids[i], e_ids)
            assert np.array_equal(d2[i], e_d2)


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_single_cell_is_exhaustive(d):
    """With one occupied cell (w larger than the range) the walk sees every point."""
    x, lab, q = wl.uniform(150, 25, d, seed=200 + d)
    g = oracle.Grid(x, lab, 4.0)
    assert g.num_cells == 1
    for k in (1, 7, 150, 160):
        ids, d2, _ = g.query(q, k)
        for i in range(q.shape[0]):
            e_ids, e_d2 = refs.knn_exhaustive(x, q[i], k)
            assert np.array_equal(ids[i], e_ids)
            assert np.array_equal(d2[i], e_d2)


@pytest.mark.parametrize("d,w", [(2, 0.07), (3, 0.2), (4, 0.3)])
def test_no_stop_rule_is_exhaustive(d, w):
    """Without the stop rule the walk ends only when the box is covered: exact KNN."""
    x, lab, q = wl.uniform(400, 30, d, seed=300 + d)
    q = np.concatenate([q, np.array([[-1.5] * d, [2.5] * d], np.float32)])
    g = oracle.Grid(x, lab, w)
    for k in (1, 9):
        for i in range(q.shape[0]):
            ids, d2, _, _ = g.query_one(q[i], k, stop_rule=False)
            e_ids, e_d2 = refs.knn_exhaustive(x, q[i], k)
            assert np.array_equal(ids, e_ids)
            assert np.array_equal(d2, e_d2)


# ---- the stop rule, restated on sets ----

def _p1_cases():
    out = []
    for d, n, w, k, seed in [(1, 200, 0.02, 3, 1), (2, 300, 0.05, 5, 2), (2, 300, 0.013, 4, 3),
                             (3, 400, 0.15, 7, 4), (4, 300, 0.35, 3, 5), (6, 200, 0.6, 2, 6)]:
        out.append((d, n, w, k, seed))
    return out


@pytest.mark.parametrize("d,n,w,k,seed", _p1_cases())
def test_stop_rule_set_form(d, n, w, k, seed):
    """The walk's result and depth equal the set form of the stop rule (Sec. III.B)."""
    x, lab, q = wl.uniform(n, 40, d, seed=seed)
    q = np.concatenate([q, np.array([[-0.5] * d, [1.7] * d, [0.5] * d], np.float32)])
    g = oracle.Grid(x, lab, w)
    pc = g.cells_of(x)
    cmax = g.origin()[1]
    for i in range(q.shape[0]):
        c0 = g.cells_of(q[i][None], as_query=True)[0]
        e_ids, e_d2, lstar = refs.set_form(x, pc, q[i], c0, cmax, k)
        ids, d2, _, st = g.query_one(q[i], k)
        assert np.array_equal(ids, e_ids), (i, ids, e_ids)
        assert np.array_equal(d2, e_d2)
        assert st[0] == lstar + 1
        # cells looked up and points examined are those of cube(L*)
        inside = np.abs(pc - c0).max(axis=1) <= lstar
        assert st[2] == inside.sum()
        assert st[1] == len({tuple(c) for c in pc[inside].tolist()})


def test_stop_rule_lattice_ties():
    """Integer lattice: many exact distance ties, broken by the lower training index."""
    x, lab, q = wl.lattice(9, 2, 60, seed=11)
    g = oracle.Grid(x, lab, 1.0)
    pc = g.cells_of(x)
    cmax = g.origin()[1]
    for k in (1, 4, 9, 13):
        for i in range(q.shape[0]):
            c0 = g.cells_of(q[i][None], as_query=True)[0]
            e_ids, e_d2, lstar = refs.set_form(x, pc, q[i], c0, cmax, k)
            ids, d2, _, st = g.query_one(q[i], k)
            assert np.array_equal(ids, e_ids)
            assert np.array_equal(d2, e_d2)
            assert st[0] == lstar + 1


def test_fewer_points_than_k():
    x, lab, q = wl.uniform(6, 4, 2, seed=9)
    g = oracle.Grid(x, lab, 0.1)
    ids, d2, pred = g.query(q, 10, 0)
    for i in range(q.shape[0]):
        e_ids, e_d2 = refs.knn_exhaustive(x, q[i], 10)
        assert np.array_equal(ids[i], e_ids)
        assert (ids[i, 6:] == -1).all() and np.isinf(d2[i, 6:]).all()
        assert pred[i] == refs.vote(lab[ids[i, :6]])


def test_no_fma_in_distance():
    """Squared distance is a sum of rounded products: a fused multiply-add differs here."""
    rng = np.random.default_rng(1234)
    for _ in range(10000):
        p = rng.random(2).astype(np.float32)
        q = rng.random(2).astype(np.float32)
        t = (q - p).astype(np.float32)
        unfused = np.float32(np.float32(t[0] * t[0]) + np.float32(t[1] * t[1]))
        fused = np.float32(np.float64(np.float32(t[0] * t[0])) + np.float64(t[1]) * np.float64(t[1]))
        if unfused != fused:
            break
    else:
        pytest.fail("no distinguishing case found")
    x = np.stack([p, p + 10]).astype(np.float32)
    g = oracle.Grid(x, np.zeros(2, np.int32), 100.0)
    _, d2, _, _ = g.query_one(q, 1)
    assert d2[0] == unfused and d2[0] != fused


# ---- prediction (Sec. I, Sec. III.D) ----

def test_vote_single_class_and_constant_mean():
    x, _, q = wl.uniform(500, 30, 3, seed=21)
    g = oracle.Grid(x, np.full(500, 7, np.int32), 0.15)
    _, _, pred = g.query(q, 9, 0)
    assert (pred == 7).all()
    g2 = oracle.Grid(x, np.full(500, 2.375, np.float32), 0.15)
    _, _, pred2 = g2.query(q, 9, 1)
    assert (pred2 == np.float32(2.375)).all()


def test_vote_tie_goes_to_smallest_label():
    # four points at distances 1, 2, 3, 4 from the query (w large: one cell)
    x = np.array([[1.0], [2.0], [3.0], [4.0], [50.0]], np.float32)
    q = np.array([[0.0]], np.float32)
    for labels, k, expect in [([5, 3, 5, 3, 0], 4, 3), ([2, 9, 9, 2, 0], 4, 2),
                              ([4, 1, 1, 4, 0], 3, 1), ([8, 6, 7, 5, 0], 4, 5),
                              ([-3, 2, 2, -3, 0], 4, -3)]:
        g = oracle.Grid(x, np.array(labels, np.int32), 100.0)
        _, _, pred = g.query(q, k, 0)
        assert pred[0] == expect, (labels, k)
        assert refs.vote(np.array(labels[:k])) == expect


def test_mean_of_known_values():
    x = np.array([[1.0], [2.0], [3.0], [4.0], [50.0]], np.float32)
    y = np.array([1.0, 2.0, 3.0, 4.0, 1000.0], np.float32)
    g = oracle.Grid(x, y, 100.0)
    _, _, pred = g.query(np.array([[0.0]], np.float32), 4, 1)
    assert pred[0] == np.float32(2.5)
    _, _, pred = g.query(np.array([[0.0]], np.float32), 3, 1)
    assert pred[0] == np.float32(2.0)
    # 0.1 + 0.2 + 0.3 in double, divided by 3, then rounded to float32
    y2 = np.array([0.1, 0.2, 0.3, 9.0, 9.0], np.float32)
    g2 = oracle.Grid(x, y2, 100.0)
    _, _, pred = g2.query(np.array([[0.0]], np.float32), 3, 1)
    s = float(np.float32(0.1)) + float(np.float32(0.2)) + float(np.float32(0.3))
    assert pred[0] == np.float32(s / 3.0)


def test_bad_arguments():
    x = np.zeros((3, 2), np.float32)
    with pytest.raises(ValueError):
        oracle.Grid(x, None, 0.0)
    with pytest.raises(ValueError):
        oracle.Grid(x, None, float("inf"))
    bad = x.copy()
    bad[1, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.Grid(bad, None, 1.0)
    with pytest.raises(ValueError):
        oracle.Grid(np.zeros((3, 9), np.float32), None, 1.0)


def test_mean_with_fewer_points_than_k():
    """Fewer than k points: the mean is over the ones found."""
    x = np.array([[1.0], [2.0], [4.0]], np.float32)
    y = np.array([1.0, 2.0, 6.0], np.float32)
    g = oracle.Grid(x, y, 0.5)
    ids, _, pred = g.query(np.array([[0.0]], np.float32), 5, 1)
    assert ids[0].tolist() == [0, 1, 2, -1, -1]
    assert pred[0] == np.float32(3.0)


def test_mean_sums_in_double():
    """The mean sums in double precision: 2^24 + 1 - 2^24 keeps the 1 (float would lose it)."""
    x = np.array([[1.0], [2.0], [3.0]], np.float32)
    y = np.array([16777216.0, 1.0, -16777216.0], np.float32)
    g = oracle.Grid(x, y, 100.0)
    _, _, pred = g.query(np.array([[0.0]], np.float32), 3, 1)
    assert pred[0] == np.float32(1.0 / 3.0)


# ---- median head (Sec. I and Sec. III.D name the median beside the average) ----

def _one_dim_grid(y):
    x = np.arange(1, len(y) + 1, dtype=np.float32).reshape(-1, 1)  # distances 1, 2, ... from 0
    return oracle.Grid(x, np.asarray(y, np.float32), 1000.0)


def test_median_of_known_values():
    g = _one_dim_grid([5.0, -1.0, 3.0, 2.0, 1000.0])
    q = np.array([[0.0]], np.float32)
    for k, expect in [(1, 5.0), (2, 2.0), (3, 3.0), (4, 2.5), (5, 3.0)]:
        _, _, pred = g.query(q, k, 2)
        assert pred[0] == np.float32(expect), k


def test_median_matches_statistics_median():
    """Against Python's statistics.median of the outputs of the neighbours the walk found."""
    import statistics

    for seed, (n, d, k, w) in enumerate([(300, 2, 5, 0.1), (300, 3, 8, 0.2), (40, 1, 7, 0.05),
                                         (200, 4, 32, 0.3), (5, 2, 9, 0.5)]):
        x, _, q = wl.uniform(n, 20, d, seed=100 + seed)
        rng = np.random.default_rng(seed)
        y = rng.integers(-4, 5, size=n).astype(np.float32) * np.float32(0.75)  # many equal outputs
        g = oracle.Grid(x, y, w)
        ids, _, pred = g.query(q, k, 2)
        for i in range(q.shape[0]):
            vals = [float(y[j]) for j in ids[i] if j >= 0]
            assert pred[i] == np.float32(statistics.median(vals)), (seed, i)


def test_median_signed_zero_by_total_order():
    """-0 sorts before +0: the middle of {+0, -0, -0} is -0, of {-0, +0, +0} is +0."""
    q = np.array([[0.0]], np.float32)
    _, _, pred = _one_dim_grid([0.0, -0.0, -0.0]).query(q, 3, 2)
    assert pred.view(np.uint32)[0] == 0x80000000
    _, _, pred = _one_dim_grid([-0.0, 0.0, 0.0]).query(q, 3, 2)
    assert pred.view(np.uint32)[0] == 0
    # zeros met in the order +0, -0: sorted -0, +0 whatever the neighbour order
    _, _, pred = _one_dim_grid([0.0, -0.0, 1.0]).query(q, 3, 2)
    assert pred.view(np.uint32)[0] == 0
    _, _, pred = _one_dim_grid([0.0, -0.0, -1.0]).query(q, 3, 2)
    assert pred.view(np.uint32)[0] == 0x80000000


def test_median_even_count_sums_in_double():
    """(a + b) / 2 in double: finite even where a float sum of a and b overflows."""
    a, b = np.float32(3.0e38), np.float32(3.2e38)
    _, _, pred = _one_dim_grid([a, b, 1.0, 1.0]).query(np.array([[0.0]], np.float32), 2, 2)
    assert np.isfinite(pred[0])
    assert pred[0] == np.float32((float(a) + float(b)) / 2.0)


def test_median_with_fewer_points_than_k_and_none():
    q = np.array([[0.0]], np.float32)
    _, _, pred = _one_dim_grid([4.0, 1.0, 9.0]).query(q, 6, 2)
    assert pred[0] == np.float32(4.0)


# ---- per-dimension widths, the cell measurement, the certified stop ----

def test_per_dimension_eq1_cells():
    gold = _golden("per_dim_cells.json")
    pts = np.array(gold["points"], np.float32)
    g = oracle.Grid(pts, None, np.array(gold["widths"], np.float32))
    assert g.cells_of(pts).tolist() == gold["cells"]


def _measure_brute(v):
    """Largest s whose s equal splits (Eq. 1 cells clamped to s - 1) are all occupied."""
    v = np.asarray(v, np.float32)
    lo = v.min()
    r = np.float32(v.max() - lo)
    if r == 0:
        return 1, np.float32(1.0)
    best = (1, r)
    for s in range(1, len(np.unique(v)) + 1):
        w = np.float32(r / np.float32(s))
        c = np.minimum(np.floor((v - lo) / w), s - 1).astype(np.int64)
        if set(c.tolist()) == set(range(s)):
            best = (s, w)
    return best


def test_measure_hand_examples():
    # 0..9: ten splits of width 0.9 (s = 11 leaves split 5 empty)
    x = np.arange(10, dtype=np.float32)
    # {0, 1, 3}: three splits of width 1 (3 lands in the closed last split)
    y = np.array([0, 1, 3, 0, 1, 3, 0, 1, 3, 0], np.float32)
    # {0, 1, 2, 10}: s = 4 (width 2.5) and s = 3 leave middle splits empty; s = 2
    z = np.array([0, 1, 2, 10, 0, 1, 2, 10, 0, 1], np.float32)
    splits, widths = oracle.measure_cells(np.stack([x, y, z], axis=1))
    assert splits.tolist() == [10, 3, 2]
    assert widths.tolist() == [np.float32(0.9), 1.0, 5.0]


@pytest.mark.parametrize("seed", range(6))
def test_measure_is_the_largest_full_split_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, d = int(rng.integers(5, 120)), int(rng.integers(1, 4))
    if seed % 3 == 0:
        x = rng.random((n, d))
    elif seed % 3 == 1:
        x = np.round(rng.normal(0.5, 0.2, (n, d)) * 20) / 20  # ties and gaps
    else:
        x = np.concatenate([rng.normal(0.2, 0.01, (n, d)), rng.normal(0.9, 0.05, (5, d))])
    x = x.astype(np.float32)
    splits, widths = oracle.measure_cells(x)
    for j in range(x.shape[1]):
        s, w = _measure_brute(x[:, j])
        assert splits[j] == s and widths[j] == w, (j, splits[j], s)


def test_measured_grid_occupies_every_split():
    x, _, _ = wl.uniform(400, 1, 3, seed=77)
    splits, widths = oracle.measure_cells(x)
    g = oracle.Grid(x, None, widths, splits=splits)
    coords, counts, _ = g.cells()
    assert counts.sum() == 400
    for j in range(3):
        assert sorted(set(coords[:, j].tolist())) == list(range(int(splits[j])))


def _exhaustive(x, q, k):
    rows = [refs.knn_exhaustive(x, qi, k) for qi in q]
    return np.stack([r[0] for r in rows]), np.stack([r[1] for r in rows])


def _exact_cases():
    out = []
    for seed, (n, d, w) in enumerate([(500, 2, 0.05), (800, 3, 0.11), (300, 4, 0.2),
                                      (400, 1, 0.01), (250, 6, 0.4)]):
        x, _, q = wl.uniform(n, 40, d, seed=600 + seed)
        q = np.concatenate([q, np.full((2, d), -0.3), np.full((1, d), 1.7)]).astype(np.float32)
        out.append((x, q, w, None))
    # clustered points, per-dimension widths
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(0.3, 0.02, (300, 3)), rng.random((100, 3))]).astype(np.float32)
    out.append((x, rng.random((40, 3)).astype(np.float32), np.float32([0.05, 0.02, 0.1]), None))
    # lattice with exact ties
    xl, _, ql = wl.lattice(12, 2, 40, seed=3)
    out.append((xl, ql, 1.0, None))
    return out


@pytest.mark.parametrize("k", [1, 5, 16])
def test_exact_rule_equals_exhaustive_knn(k):
    for x, q, w, splits in _exact_cases():
        g = oracle.Grid(x, None, w, splits=splits)
        ids, d2, _ = g.query(q, k, -1, rule=oracle.RULE_EXACT)
        e_ids, e_d2 = _exhaustive(x, q, k)
        assert np.array_equal(ids, e_ids)
        assert np.array_equal(d2.view(np.uint32), e_d2.view(np.uint32))


def test_exact_rule_on_a_measured_grid_equals_exhaustive_knn():
    rng = np.random.default_rng(8)
    x = np.round(rng.random((600, 2)) * 50).astype(np.float32) / np.float32(50)
    splits, widths = oracle.measure_cells(x)
    g = oracle.Grid(x, None, widths, splits=splits)
    q = rng.random((60, 2)).astype(np.float32) * np.float32(1.4) - np.float32(0.2)
    ids, d2, _ = g.query(q, 7, -1, rule=oracle.RULE_EXACT)
    e_ids, e_d2 = _exhaustive(x, q, 7)
    assert np.array_equal(ids, e_ids)
    assert np.array_equal(d2.view(np.uint32), e_d2.view(np.uint32))


def test_exact_rule_stops_once_certified():
    """On a unit lattice with w = 1 and k = 1, a query at a lattice point has
    its neighbour at distance 0 in the central cell; the gap to the cells
    beyond cube(1) is at least 1, so the walk stops after layer 1 (2 layers),
    long before covering the 40 x 40 box."""
    xl = np.stack(np.meshgrid(np.arange(40), np.arange(40)), -1).reshape(-1, 2).astype(np.float32)
    g = oracle.Grid(xl, None, 1.0)
    q = np.array([[20.0, 20.0], [7.0, 31.0]], np.float32)
    _, _, _, st = g.query(q, 1, -1, stats=True, rule=oracle.RULE_EXACT)
    assert st[:, 0].tolist() == [2, 2]
    _, _, _, st0 = g.query(q, 1, -1, stats=True, rule=oracle.RULE_NONE)
    assert (st0[:, 0] > 10).all()
    # by the upper edge of the box no cell lies above, so only the other sides
    # bound the unseen points: nearest (39, 20) at 0.95^2 + 0.5^2 = 1.1525,
    # below the gap 1.5^2 left after layer 1 (dimension 1, both sides)
    _, _, _, st = g.query(np.array([[39.95, 20.5]], np.float32), 1, -1, stats=True,
                          rule=oracle.RULE_EXACT)
    assert st[0, 0] == 2


def test_recall_is_reported_and_exact_when_one_cell_holds_everything():
    """Recall of the paper's rule against exhaustive KNN (reported, not pinned):
    a value in [0, 1]; exactly 1 when a single cell holds every point."""
    x, lab, q = wl.uniform(800, 60, 3, seed=31)
    r, dr = oracle.recall(oracle.Grid(x, lab, 0.08), x, q, 10)
    assert 0.0 <= r <= 1.0 and 0.0 <= dr <= 1.0 and dr >= r - 1e-12
    assert oracle.recall(oracle.Grid(x, lab, 10.0), x, q, 10) == (1.0, 1.0)
