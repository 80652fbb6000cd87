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


# problems of the 256-problem batched workload: the heaviest d=6 one (problem
# 100, n = 1,382,810, k = 15), the largest of each dimension, and k = 32 ones
# from 1,432 to 1,864,855 points
_FULL_SUBSET = [100, 206, 9, 20, 38, 199, 107, 12, 1, 7, 23, 57, 44]


def test_full_size_batched_subset_matches_the_oracle():
    """A subset of the real batched workload in one batch, with the
    autotuner's widths, in the bench's launch configuration: a seeded sample
    of each problem's queries equals the oracle element by element, and every
    query equals the plain form."""
    from paper_2004_02290_gb300 import autotune

    ps = wl.gen_batched(256, seed=3)
    sub = [ps[i] for i in _FULL_SUBSET]
    dev = torch.device("cuda:0")
    widths = [autotune.tune_width(p.points, p.labels, p.queries, p.k, p.mode, dev=dev).width
              for p in sub]
    b = knn.knn_batch_build([_dev(p.points) for p in sub], [_dev(p.labels) for p in sub],
                            widths)
    bids, bd2, bpred = b.query([_dev(p.queries) for p in sub], [p.k for p in sub],
                               [p.mode for p in sub], flags=knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    b.free()
    rng = np.random.default_rng(2024)
    for j, (p, w) in enumerate(zip(sub, widths)):
        ids, d2, pred = bids[j].cpu().numpy(), bd2[j].cpu().numpy(), bpred[j].cpu().numpy()
        pick = np.sort(rng.choice(p.m, size=min(p.m, 300), replace=False))
        g = oracle.Grid(p.points, p.labels, w)
        e_ids, e_d2, e_pred = g.query(p.queries[pick], p.k, p.mode)
        g.close()
        where = f"problem {_FULL_SUBSET[j]} (n={p.n}, d={p.d}, k={p.k}, w={w})"
        assert np.array_equal(ids[pick], e_ids), where
        assert np.array_equal(d2[pick].view(np.uint32), e_d2.view(np.uint32)), where
        assert np.array_equal(pred[pick].view(np.uint32), e_pred.view(np.uint32)), where
        idx = knn.knn_build(_dev(p.points), _dev(p.labels), w)
        pi, pd, pp = idx.query(_dev(p.queries), p.k, p.mode, flags=knn.KNN_QUERY_CHECKED)
        torch.cuda.synchronize()
        idx.free()
        assert np.array_equal(pi.cpu().numpy(), ids), where
        assert np.array_equal(pp.cpu().numpy().view(np.uint32), pred.view(np.uint32)), where


def test_batch_with_host_buffers_matches_device_buffers():
    """knn_batch_build / knn_batch_query with host inputs and outputs
    (pinned, pageable, mixed) equal the all-device call."""
    ps, _ = _problems()
    ps = ps[:8]
    ws = [p.w for p in ps]
    ks = [p.k for p in ps]
    modes = [p.mode for p in ps]
    b = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps], ws)
    ref = b.query([_dev(p.queries) for p in ps], ks, modes, flags=knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    b.free()
    # every buffer pinned, every buffer pageable, and a mix (pinned and
    # pageable alternating over problems and arrays: copies on the side
    # stream and on the caller's stream in one call)
    # and pinned inputs with pageable outputs (the staging buffer, allocated
    # on the side stream, then also holds outputs the kernels write)
    for kind in ("pinned", "pageable", "mixed", "pinned inputs"):
        turn = [0]

        def host(a, output=False):
            t = torch.from_numpy(np.ascontiguousarray(a))
            turn[0] += 1
            pin = (kind == "pinned" or (kind == "mixed" and turn[0] % 3 != 0)
                   or (kind == "pinned inputs" and not output))
            return t.pin_memory() if pin else t
        b = knn.knn_batch_build([host(p.points) for p in ps], [host(p.labels) for p in ps], ws)
        out = ([host(np.zeros((p.m, p.k), np.int32), True) for p in ps],
               [host(np.zeros((p.m, p.k), np.float32), True) for p in ps],
               [None if p.mode < 0 else host(np.zeros(p.m, np.int32 if p.mode == knn.KNN_VOTE
                                                      else np.float32), True) for p in ps])
        b.query([host(p.queries) for p in ps], ks, modes, flags=knn.KNN_QUERY_CHECKED, out=out)
        b.free()
        for j in range(len(ps)):
            assert np.array_equal(out[0][j].numpy(), ref[0][j].cpu().numpy())
            assert np.array_equal(out[1][j].numpy().view(np.uint32),
                                  ref[1][j].cpu().numpy().view(np.uint32))
            if out[2][j] is not None:
                assert np.array_equal(out[2][j].numpy().view(np.uint32),
                                      ref[2][j].cpu().numpy().view(np.uint32))


def test_batch_deferral_refinement_chooses_per_group():
    """The batch-level pass returns one of its options for every kernel group,
    applied to all of the group's problems, and leaves phase timing off."""
    from paper_2004_02290_gb300 import autotune

    ps, _ = _problems()
    ps = ps[:8]
    start = [(0, -1)] * len(ps)
    got, sec, groups = autotune.refine_batch_deferral(ps, [p.w for p in ps], start, reps=1)
    assert sec > 0 and groups and len(got) == len(ps)
    assert all(g.startswith("query.d") for g in groups)
    options = {"per problem": (0, -1), "default": (0, 0), "none": (-1, -1)}
    assert set(groups.values()) <= set(options)
    for i, p in enumerate(ps):
        assert tuple(got[i]) in options.values()
    b = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps],
                            [p.w for p in ps])
    # every problem of a group got its group's option
    members = {}
    for i, p in enumerate(ps):
        dense = b.info(i).table == knn.KNN_TABLE_DENSE
        g = f"query.d{p.d}.{'k64' if p.k > 32 else 'k32'}.{'dense' if dense else 'hash'}"
        members.setdefault(g, set()).add(tuple(got[i]))
    assert set(members) == set(groups)
    for g, opts in members.items():
        assert opts == {options[groups[g]]}
    b.query([_dev(p.queries) for p in ps], [p.k for p in ps], [p.mode for p in ps])
    torch.cuda.synchronize()
    b.free()
    assert knn.knn_timing_read() == []


_ALLOC_FAIL = r"""
import numpy as np, torch, sys
sys.path.insert(0, %r)
from paper_2004_02290_gb300 import knn, workloads as wl
ps = wl.gen_batched(6, seed=5, n_lo=300, n_hi=5000, dims=(2, 3, 6), ks=(1, 5, 15))
ws = [float(np.float32(0.08 * p.d / 3.0)) for p in ps]
pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
def run():
    b = knn.knn_batch_build([pin(p.points) for p in ps], [pin(p.labels) for p in ps], ws)
    try:
        out = ([pin(np.zeros((p.m, p.k), np.int32)) for p in ps],
               [pin(np.zeros((p.m, p.k), np.float32)) for p in ps],
               [pin(np.zeros(p.m, np.int32 if p.mode == knn.KNN_VOTE else np.float32))
                for p in ps])
        b.query([pin(p.queries) for p in ps], [p.k for p in ps], [p.mode for p in ps],
                flags=knn.KNN_QUERY_CHECKED, out=out)
        return out
    finally:
        b.free()
try:
    run()
    print("NOFAIL")
except knn.KnnError as e:
    print("CODE", e.code)
# the next build and query work and match the device-buffer path
got = run()
b = knn.knn_batch_build([torch.from_numpy(p.points).cuda() for p in ps],
                        [torch.from_numpy(p.labels).cuda() for p in ps], ws)
ref = b.query([torch.from_numpy(p.queries).cuda() for p in ps], [p.k for p in ps],
              [p.mode for p in ps])
torch.cuda.synchronize()
b.free()
ok = all(np.array_equal(got[0][i].numpy(), ref[0][i].cpu().numpy()) for i in range(len(ps)))
print("AFTER", "same" if ok else "differ")
"""


def test_batch_host_buffers_survive_allocation_failure():
    """An allocation that fails at a point of a batched build or query on
    pinned host buffers (with copies on the side stream in flight) returns
    KNN_ENOMEM, and the next call works and matches the device-buffer path."""
    codes = []
    for at in ("1", "3", "6", "10", "15", "20"):
        env = dict(os.environ, GHN_FAIL_ALLOC_AT=at)
        r = subprocess.run([sys.executable, "-c", _ALLOC_FAIL % ROOT], cwd=ROOT, env=env,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, (at, r.stderr[-2000:])
        assert "AFTER same" in r.stdout, (at, r.stdout)
        codes.append(r.stdout.split()[1] if r.stdout.startswith("CODE") else "none")
    assert codes.count("2") >= 4, codes  # KNN_ENOMEM at most of the points


def test_batch_pinned_inputs_on_a_user_stream():
    """Pinned host inputs on a non-default stream: the build is still running
    on that stream when the query's staging copies start on the library's
    side stream.  Each call returns only once its host inputs have been read,
    so overwriting them right after the call changes nothing; the results
    equal the device-buffer call's."""
    ps, _ = _problems()
    ps = ps[:8]
    ws = [p.w for p in ps]
    ks = [p.k for p in ps]
    modes = [p.mode for p in ps]
    b = knn.knn_batch_build([_dev(p.points) for p in ps], [_dev(p.labels) for p in ps], ws)
    ref = b.query([_dev(p.queries) for p in ps], ks, modes, flags=knn.KNN_QUERY_CHECKED)
    torch.cuda.synchronize()
    b.free()
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    s = torch.cuda.Stream()
    for rep in range(2):
        pts = [pin(p.points) for p in ps]
        lab = [pin(p.labels) for p in ps]
        b = knn.knn_batch_build(pts, lab, ws, stream=s)
        for t in pts + lab:
            t.view(torch.int32).fill_(-7)  # the build has read them
        qs = [pin(p.queries) for p in ps]
        got = ([torch.empty((p.m, p.k), dtype=torch.int32, device="cuda") for p in ps],
               [torch.empty((p.m, p.k), dtype=torch.float32, device="cuda") for p in ps],
               [None if p.mode < 0 else
                torch.empty(p.m, dtype=torch.int32 if p.mode == knn.KNN_VOTE else torch.float32,
                            device="cuda") for p in ps])
        # device outputs: nothing in the call waits for the kernels
        b.query(qs, ks, modes, stream=s, out=got)
        for t in qs:
            t.fill_(float("nan"))  # the query has read them
        s.synchronize()
        b.free()
        for j in range(len(ps)):
            assert np.array_equal(got[0][j].cpu().numpy(), ref[0][j].cpu().numpy()), (rep, j)
            assert np.array_equal(got[1][j].cpu().numpy().view(np.uint32),
                                  ref[1][j].cpu().numpy().view(np.uint32)), (rep, j)
            if got[2][j] is not None:
                assert np.array_equal(got[2][j].cpu().numpy().view(np.uint32),
                                      ref[2][j].cpu().numpy().view(np.uint32)), (rep, j)
