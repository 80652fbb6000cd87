"""Property tests of the oracle (random shapes, widths, ties, duplicates).

Each property is a fact that the paper or the mathematics fixes, checked on
inputs that hypothesis draws:
* without the stop rule the walk visits every occupied cell, so it equals
  exhaustive KNN (Sec. I);
* the certified stop equals exhaustive KNN, on grids with per-dimension widths;
* the paper's rule returns k points whenever n >= k, all of them at or beyond
  the exact neighbours' distances, and the exact k-th distance is no larger
  than its own;
* the cell measurement is the largest split count whose splits are all
  occupied (Sec. III.A), by brute force over every count.
"""
import numpy as np
import pytest

import oracle
from tests import refs

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies
given, settings = hypothesis.given, hypothesis.settings


def _exhaustive(x, q, k):
    rows = [refs.knn_exhaustive(x, qi, k) for qi in q]
    return np.stack([r[0] for r in rows]), np.stack([r[1] for r in rows])


@st.composite
def problems(draw):
    d = draw(st.integers(1, 4))
    n = draw(st.integers(1, 60))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    grid = draw(st.sampled_from([0, 8, 32]))  # 0: continuous; else values on a lattice (ties)
    x = rng.random((n, d))
    if grid:
        x = np.round(x * grid) / grid
    if n > 3 and draw(st.booleans()):
        x[1] = x[0]  # a duplicate point
    q = rng.random((draw(st.integers(1, 6)), d)) * 1.4 - 0.2
    widths = np.asarray([draw(st.sampled_from([0.03, 0.07, 0.15, 0.4, 2.0])) for _ in range(d)])
    k = draw(st.integers(1, 12))
    return x.astype(np.float32), q.astype(np.float32), widths.astype(np.float32), k


@settings(max_examples=120, deadline=None)
@given(problems())
def test_walk_without_stop_rule_is_exhaustive(p):
    x, q, w, k = p
    g = oracle.Grid(x, None, w)
    ids, d2, _ = g.query(q, k, -1, rule=oracle.RULE_NONE)
    e_ids, e_d2 = _exhaustive(x, q, k)
    assert np.array_equal(ids, e_ids)
    assert np.array_equal(d2.view(np.uint32), e_d2.view(np.uint32))


@settings(max_examples=120, deadline=None)
@given(problems())
def test_certified_stop_is_exhaustive(p):
    x, q, w, k = p
    g = oracle.Grid(x, None, w)
    ids, d2, _ = g.query(q, k, -1, rule=oracle.RULE_EXACT)
    e_ids, e_d2 = _exhaustive(x, q, k)
    assert np.array_equal(ids, e_ids)
    assert np.array_equal(d2.view(np.uint32), e_d2.view(np.uint32))


@settings(max_examples=120, deadline=None)
@given(problems())
def test_paper_rule_returns_k_and_never_beats_exact(p):
    x, q, w, k = p
    g = oracle.Grid(x, None, w)
    ids, d2, _ = g.query(q, k, -1)
    e_ids, e_d2 = _exhaustive(x, q, k)
    found = (ids >= 0).sum(axis=1)
    assert (found == min(k, x.shape[0])).all()
    # the i-th returned distance is never below the i-th exact one
    assert (d2 >= e_d2).all()


@settings(max_examples=80, deadline=None)
@given(st.integers(1, 80), st.integers(0, 2**31 - 1), st.sampled_from([0, 5, 20, 100]))
def test_measurement_is_the_largest_full_split(n, seed, grid):
    rng = np.random.default_rng(seed)
    v = rng.random(n)
    if grid:
        v = np.round(v * grid) / grid
    v = v.astype(np.float32)
    splits, widths = oracle.measure_cells(v.reshape(-1, 1))
    lo = v.min()
    r = np.float32(v.max() - lo)
    if r == 0:
        assert (splits[0], widths[0]) == (1, np.float32(1.0))
        return
    best = None
    for s in range(1, len(np.unique(v)) + 1):
        w = np.float32(r / np.float32(s))
        c = np.minimum(np.floor((v - lo) / w), s - 1).astype(np.int64)
        if set(c.tolist()) == set(range(s)):
            best = (s, w)
    assert (int(splits[0]), widths[0]) == best
