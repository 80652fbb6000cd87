"""The batched form (many indexes in one build pass and one query launch per
dimension) against the plain form (knn_build + knn_query per index) and the
oracle, through the C ABI (GPU needed).  Outputs must be identical."""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _problems():
    """Uneven problems over every dimension, k up to 64, every head and both tables."""
    ps = wl.gen_batched(20, seed=11, n_lo=300, n_hi=30_000, dims=(1, 2, 3, 4, 5, 6, 7, 8),
                        ks=(1, 5, 15, 32, 40, 64))
    tables = []
    rng = np.random.default_rng(2)
    for i, p in enumerate(ps):
        p.w = float(np.float32(0.05 * (1.0 + (i % 4)) * (p.d / 3.0)))
        tables.append(int(rng.choice([knn.KNN_TABLE_AUTO, knn.KNN_TABLE_HASH])))
        if i % 4 == 3:
            p.mode = knn.KNN_MEDIAN  # a regression problem with the median head
    # a problem with far queries and one with a single occupied cell
    ps[3].queries[:3] = np.float32(40.0)
    ps[5].w = 1000.0
    return ps, tables


def _plain(ps, tables):
    out = []
    for p, t in zip(ps, tables):
        idx = knn.knn_build(_dev(p.points), _dev(p.labels), p.w, t)
        ids, d2, pred = idx.query(_dev(p.queries), p.k, p.mode, flags=knn.KNN_QUERY_CHECKED)
        torch.cuda.synchronize()
        out.append((ids.cpu().numpy(), d2.cpu().numpy(), pred.cpu().numpy()))
        idx.free()
    return out


def _same(a, b):
    for x, y in zip(a, b):
        assert x.shape == y.shape
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def test_batch_equals_plain_and_oracle():
    ps, tables = _problems()
    batch = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps],
                                [p.w for p in ps], tables)
    ids, d2, pred = batch.query([_dev(p.queries) for p in ps], [p.k for p in ps],
                                [p.mode for p in ps], flags=knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    plain = _plain(ps, tables)
    for i, p in enumerate(ps):
        got = (ids[i].cpu().numpy(), d2[i].cpu().numpy(), pred[i].cpu().numpy())
        _same(got, plain[i])
        inf = batch.info(i)
        assert inf.n == p.n and inf.d == p.d
        if tables[i] == knn.KNN_TABLE_HASH:
            assert inf.table == knn.KNN_TABLE_HASH
    for i in (0, 3, 5, 9, 14):
        p = ps[i]
        e = oracle.Grid(p.points, p.labels, p.w).query(p.queries, p.k, p.mode)
        _same((ids[i].cpu().numpy(), d2[i].cpu().numpy(), pred[i].cpu().numpy()), e)
    batch.free()


def test_batch_plan_graph_replays():
    ps, tables = _problems()
    batch = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps],
                                [p.w for p in ps], tables)
    qs = [_dev(p.queries) for p in ps]
    ids, d2, pred = batch.query(qs, [p.k for p in ps], [p.mode for p in ps])
    plan, pids, pd2, ppred = batch.plan(qs, [p.k for p in ps], [p.mode for p in ps])
    for _ in range(2):
        for t in pids:
            t.fill_(-5)
        plan.run(flags=knn.KNN_QUERY_CHECKED)
        torch.cuda.synchronize()
        for i in range(len(ps)):
            assert torch.equal(pids[i], ids[i])
            assert torch.equal(pd2[i], d2[i])
            assert torch.equal(ppred[i], pred[i])
    plan.free()
    batch.free()


def test_batch_with_empty_query_sets():
    ps, tables = _problems()
    batch = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps],
                                [p.w for p in ps], tables)
    qs = [_dev(p.queries if i % 3 else p.queries[:0]) for i, p in enumerate(ps)]
    ids, d2, pred = batch.query(qs, [p.k for p in ps], [p.mode for p in ps],
                                flags=knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    plain = _plain(ps, tables)
    for i in range(len(ps)):
        if i % 3:
            _same((ids[i].cpu().numpy(), d2[i].cpu().numpy(), pred[i].cpu().numpy()), plain[i])
        else:
            assert ids[i].shape[0] == 0
    batch.free()


_FORCED = r"""
import numpy as np, torch, sys
sys.path.insert(0, %r)
from tests.test_gpu_batch import _problems, _plain, _same, _dev
from paper_2004_02290_gb300 import knn
ps, tables = _problems()
batch = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps],
                            [p.w for p in ps], tables)
ids, d2, pred = batch.query([_dev(p.queries) for p in ps], [p.k for p in ps], [p.mode for p in ps],
                            flags=knn.KNN_QUERY_CHECKED)
torch.cuda.synchronize()
plain = _plain(ps, tables)
for i in range(len(ps)):
    _same((ids[i].cpu().numpy(), d2[i].cpu().numpy(), pred[i].cpu().numpy()), plain[i])
print("OK")
"""


def test_batch_cooperative_path():
    """Every batched query forced through the cooperative kernel."""
    env = dict(os.environ, GHN_HEAVY_ROWS="2", GHN_HEAVY_CANDS="8")
    r = subprocess.run([sys.executable, "-c", _FORCED % ROOT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "OK" in r.stdout


def test_autotuner_picks_the_cheapest_candidate():
    from paper_2004_02290_gb300 import autotune

    p = wl.gen_batched(1, seed=4, n_lo=50_000, n_hi=50_001)[0]
    c = autotune.tune_width(p.points, p.labels, p.queries, p.k, p.mode)
    assert c.width in [w for w, _ in c.tried]
    assert c.est_ms == min(t for _, t in c.tried)
    assert len(c.tried) >= 3
