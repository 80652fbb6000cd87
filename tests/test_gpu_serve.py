"""Serving engine on the GPU: each result is the same alone and in the mix.

Requests against several resident indexes (d 1..6, dense and hash tables,
every head, k up to 64) are served twice: one at a time (every request in a
batch of its own) and all at once (continuous batching packs them into shared
batches).  Both must equal the oracle bit for bit (ids, squared distances,
votes, means, medians), and so must the plain knn_query of the same request.
Memory admission, drops and bad requests are covered too.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_02290_gb300 import knn
from paper_2004_02290_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


# d, n, w, table, head
INDEXES = [
    (2, 6000, 0.02, knn.KNN_TABLE_DENSE, knn.KNN_VOTE),
    (3, 8000, 0.05, knn.KNN_TABLE_HASH, knn.KNN_MEAN),
    (4, 5000, 0.12, knn.KNN_TABLE_AUTO, knn.KNN_MEDIAN),
    (6, 3000, 0.35, knn.KNN_TABLE_HASH, knn.KNN_VOTE),
    (1, 2000, 0.002, knn.KNN_TABLE_AUTO, knn.KNN_MEAN),
]


def _index_data(i):
    d, n, w, table, head = INDEXES[i]
    x, lab, _ = wl.uniform(n, 1, d, seed=300 + i)
    if head != knn.KNN_VOTE:
        lab = wl.regression_targets(x, seed=i)
        if head == knn.KNN_MEDIAN:
            lab = (np.round(lab * 4) / 4).astype(np.float32)  # many equal outputs
    return x, lab


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        i = int(rng.integers(0, len(INDEXES)))
        d, _, _, _, head = INDEXES[i]
        m = int(np.exp(rng.uniform(0, np.log(400))))
        q = rng.random((m, d)).astype(np.float32) * np.float32(1.2) - np.float32(0.1)
        k = int(rng.choice([1, 5, 16, 40, 64]))
        mode = head if rng.random() < 0.8 else knn.KNN_NONE
        reqs.append((i, q, k, mode))
    return reqs


def _serve(srv, ids_of, reqs, together):
    out = [None] * len(reqs)
    infos = [None] * len(reqs)
    if together:
        tickets = [srv.submit(ids_of[i], q, k, mode) for (i, q, k, mode) in reqs]
        for j, (t, ids, d2, pred) in enumerate(tickets):
            infos[j] = srv.wait(t)
            out[j] = (ids, d2, pred)
    else:
        for j, (i, q, k, mode) in enumerate(reqs):
            t, ids, d2, pred = srv.submit(ids_of[i], q, k, mode)
            infos[j] = srv.wait(t)
            out[j] = (ids, d2, pred)
    return out, infos


def _same(a, b):
    ids, d2, pred = a
    e_ids, e_d2, e_pred = b
    assert np.array_equal(ids, e_ids)
    assert np.array_equal(d2.view(np.uint32), e_d2.view(np.uint32))
    if e_pred is None:
        assert pred is None
    else:
        assert np.array_equal(np.asarray(pred).view(np.uint32), np.asarray(e_pred).view(np.uint32))


@pytest.fixture(scope="module")
def server_with_indexes():
    srv = knn.Server(max_inflight=2, max_batch_queries=8192, max_batch_requests=64)
    data = [_index_data(i) for i in range(len(INDEXES))]
    ids_of = []
    for i, (x, lab) in enumerate(data):
        d, n, w, table, head = INDEXES[i]
        iid, t = srv.build(x, lab, w, table)
        ids_of.append(iid)
        assert srv.wait(t).status == knn.KNN_OK
    yield srv, ids_of, data
    srv.close()


def test_alone_equals_mixed_equals_oracle(server_with_indexes):
    srv, ids_of, data = server_with_indexes
    reqs = _requests(70, seed=1)
    alone, ainfo = _serve(srv, ids_of, reqs, together=False)
    mixed, minfo = _serve(srv, ids_of, reqs, together=True)
    assert all(i.status == knn.KNN_OK for i in ainfo + minfo)
    # alone: one batch per request; mixed: requests shared batches
    assert len({i.batch for i in ainfo}) == len(reqs)
    assert len({i.batch for i in minfo}) < len(reqs)
    grids = [oracle.Grid(x, lab, INDEXES[i][2]) for i, (x, lab) in enumerate(data)]
    for j, (i, q, k, mode) in enumerate(reqs):
        _same(alone[j], mixed[j])
        e_ids, e_d2, e_pred = grids[i].query(q, k, mode)
        _same(mixed[j], (e_ids, e_d2, e_pred))


def test_served_equals_plain_query(server_with_indexes):
    srv, ids_of, data = server_with_indexes
    reqs = _requests(12, seed=2)
    mixed, _ = _serve(srv, ids_of, reqs, together=True)
    plain = {}
    for j, (i, q, k, mode) in enumerate(reqs):
        if i not in plain:
            x, lab = data[i]
            plain[i] = knn.knn_build(torch.from_numpy(x).cuda(), torch.from_numpy(lab).cuda(),
                                     INDEXES[i][2], INDEXES[i][3])
        ids, d2, pred = plain[i].query(q, k, mode, flags=knn.KNN_QUERY_CHECKED)
        _same(mixed[j], (np.asarray(ids), np.asarray(d2), None if pred is None else np.asarray(pred)))
    for idx in plain.values():
        idx.free()


def test_non_finite_query_fails_only_its_request(server_with_indexes):
    srv, ids_of, data = server_with_indexes
    good = np.full((3, 2), 0.5, np.float32)
    bad = good.copy()
    bad[1, 0] = np.nan
    t1, ids1, _, _ = srv.submit(ids_of[0], good, 5, knn.KNN_VOTE)
    t2, ids2, _, _ = srv.submit(ids_of[0], bad, 5, knn.KNN_VOTE)
    i1, i2 = srv.wait(t1), srv.wait(t2)
    assert i1.status == knn.KNN_OK
    assert i2.status == knn.KNN_EINVAL
    assert (ids2[1] == -1).all()
    assert np.array_equal(ids2[0], ids1[0])


def test_empty_and_oversized_requests(server_with_indexes):
    srv, ids_of, _ = server_with_indexes
    t, ids, _, _ = srv.submit(ids_of[1], np.zeros((0, 3), np.float32), 4)
    assert srv.wait(t).status == knn.KNN_OK
    with pytest.raises(knn.KnnError):
        srv.submit(ids_of[1], np.zeros((9000, 3), np.float32), 4)  # over max_batch_queries
    with pytest.raises(knn.KnnError):
        srv.submit(12345, np.zeros((1, 3), np.float32), 4)  # unknown index
    with pytest.raises(knn.KnnError):
        srv.submit(ids_of[1], np.zeros((1, 3), np.float32), 65)


def test_memory_admission_waits_for_a_drop():
    """A budget with room for one build: the next build starts after the drop."""
    x, lab = _index_data(1)
    n, d = x.shape
    probe = knn.Server(max_inflight=1, max_batch_queries=4096, max_batch_requests=16)
    buffers = probe.stats().buffer_bytes
    probe.close()
    bound = knn.knn_server_build_bytes(n, d, True)
    srv = knn.Server(memory_budget=buffers + bound + 1024, max_inflight=1,
                     max_batch_queries=4096, max_batch_requests=16)
    try:
        a, ta = srv.build(x, lab, 0.05)
        b, tb = srv.build(x, lab, 0.05)
        assert srv.wait(ta).status == knn.KNN_OK
        # b cannot start while a is resident
        assert srv.wait(tb, timeout_us=200_000) is None
        s = srv.stats()
        assert s.waiting_builds == 1 and s.resident_bytes > 1024
        # queries against b wait for its build; queries against a still run
        q = np.random.default_rng(0).random((50, 3)).astype(np.float32)
        tqb, ids_b, d2_b, pred_b = srv.submit(b, q, 7, knn.KNN_MEAN)
        tqa, ids_a, d2_a, pred_a = srv.submit(a, q, 7, knn.KNN_MEAN)
        assert srv.wait(tqa).status == knn.KNN_OK
        assert srv.test(tqb) is None
        td = srv.drop(a)
        info_d = srv.wait(td)
        info_b = srv.wait(tb)
        assert info_b.status == knn.KNN_OK
        assert info_b.t_dispatch_ns >= info_d.t_done_ns
        assert srv.wait(tqb).status == knn.KNN_OK
        _same((ids_b, d2_b, pred_b), (ids_a, d2_a, pred_a))
        with pytest.raises(knn.KnnError):
            srv.submit(a, q, 7)  # dropped
        # a build that could never fit fails at once
        with pytest.raises(knn.KnnError) as e:
            srv.build(np.zeros((4 * n, 3), np.float32), None, 0.05)
        assert e.value.code == knn.KNN_ENOMEM
    finally:
        srv.close()


def test_drop_waits_for_earlier_requests(server_with_indexes):
    srv, _, _ = server_with_indexes
    x, lab = _index_data(0)
    iid, t = srv.build(x, lab, 0.02)
    q = np.random.default_rng(3).random((200, 2)).astype(np.float32)
    reqs = [srv.submit(iid, q, 9, knn.KNN_VOTE) for _ in range(10)]  # may queue behind the build
    td = srv.drop(iid)
    assert srv.wait(t).status == knn.KNN_OK
    done = [srv.wait(r[0]) for r in reqs]
    assert all(i.status == knn.KNN_OK for i in done)
    info = srv.wait(td)
    assert info.status == knn.KNN_OK
    assert info.t_done_ns >= max(i.t_done_ns for i in done)
    for r in reqs[1:]:
        assert np.array_equal(r[1], reqs[0][1])


def test_borrowed_index_answers_plain_queries(server_with_indexes):
    srv, ids_of, data = server_with_indexes
    idx = srv.index(ids_of[2])
    q = np.random.default_rng(9).random((40, 4)).astype(np.float32)
    t, ids, d2, pred = srv.submit(ids_of[2], q, 11, knn.KNN_MEDIAN)
    assert srv.wait(t).status == knn.KNN_OK
    p_ids, p_d2, p_pred = idx.query(q, 11, knn.KNN_MEDIAN, flags=knn.KNN_QUERY_CHECKED)
    _same((ids, d2, pred), (np.asarray(p_ids), np.asarray(p_d2), np.asarray(p_pred)))
    idx.free()  # a no-op for a borrowed index: the server still owns it
    t, ids2, _, _ = srv.submit(ids_of[2], q, 11, knn.KNN_MEDIAN)
    assert srv.wait(t).status == knn.KNN_OK
    assert np.array_equal(ids, ids2)
    with pytest.raises(knn.KnnError):
        srv.index(987654)


def test_exact_requests_equal_exhaustive_in_the_mix(server_with_indexes):
    """Requests with the certified stop share batches with the paper's rule."""
    srv, ids_of, data = server_with_indexes
    reqs = _requests(24, seed=5)
    tickets = []
    for j, (i, q, k, mode) in enumerate(reqs):
        flags = knn.KNN_QUERY_EXACT if j % 2 else 0
        tickets.append((flags, srv.submit(ids_of[i], q, k, mode, flags=flags)))
    grids = [oracle.Grid(x, lab, INDEXES[i][2]) for i, (x, lab) in enumerate(data)]
    for (flags, (t, ids, d2, pred)), (i, q, k, mode) in zip(tickets, reqs):
        assert srv.wait(t).status == knn.KNN_OK
        rule = oracle.RULE_EXACT if flags else oracle.RULE_PAPER
        _same((ids, d2, pred), grids[i].query(q, k, mode, rule=rule))
    with pytest.raises(knn.KnnError):
        srv.submit(ids_of[0], np.zeros((1, 2), np.float32), 3, flags=knn.KNN_QUERY_SORTED)


def test_device_buffers_are_rejected(server_with_indexes):
    srv, ids_of, _ = server_with_indexes
    q = torch.zeros((4, 2), dtype=torch.float32, device="cuda")
    ids = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    t = knn.ctypes.c_int64()
    rc = knn.library().knn_server_submit(srv._h, ids_of[0], q.data_ptr(), 4, 3, -1,
                                         ids.data_ptr(), None, None, 0, knn.ctypes.byref(t))
    assert rc == knn.KNN_EINVAL


def test_submit_many_equals_single_submissions_and_is_all_or_nothing(server_with_indexes):
    srv, ids_of, data = server_with_indexes
    reqs = _requests(30, seed=8)
    many = srv.submit_many([(ids_of[i], q, k, mode) for (i, q, k, mode) in reqs])
    single, _ = _serve(srv, ids_of, reqs, together=False)
    for (t, ids, d2, pred), ref in zip(many, single):
        assert srv.wait(t).status == knn.KNN_OK
        _same((ids, d2, pred), ref)
    before = srv.stats().requests_done
    bad = [(ids_of[0], np.zeros((3, 2), np.float32), 5, knn.KNN_VOTE),
           (ids_of[0], np.zeros((3, 2), np.float32), 99, knn.KNN_VOTE)]  # k > 64
    with pytest.raises(knn.KnnError) as e:
        srv.submit_many(bad)
    assert "request 1" in str(e.value)
    assert srv.stats().requests_done == before and srv.stats().queued_requests == 0


_FAILED_BUILD = r"""
import numpy as np
from paper_2004_02290_gb300 import knn, workloads as wl
srv = knn.Server(max_inflight=1, max_batch_queries=4096, max_batch_requests=16)
x, lab, q = wl.uniform(3000, 20, 2, seed=1)
a, ta = srv.build(x, lab, 0.05)           # its first allocation fails (injected)
tq, ids, _, _ = srv.submit(a, q, 5, knn.KNN_VOTE)  # parked on the failing build
ia, iq = srv.wait(ta), srv.wait(tq)
b, tb = srv.build(x, lab, 0.05)           # the next build works
ib = srv.wait(tb)
t2, ids2, _, _ = srv.submit(b, q, 5, knn.KNN_VOTE)
i2 = srv.wait(t2)
try:
    srv.submit(a, q, 5, knn.KNN_VOTE)
    gone = False
except knn.KnnError:
    gone = True
srv.close()
print("STATUS", ia.status, iq.status, ib.status, i2.status, gone)
"""


def test_failed_build_fails_its_parked_queries_and_the_server_goes_on():
    """A build whose allocation fails (host-side injector): its ticket reports
    KNN_ENOMEM, the queries parked on it KNN_EINVAL, the index is gone, and the
    next build and its queries succeed."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, GHN_FAIL_ALLOC_AT="1", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", _FAILED_BUILD], cwd=root, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    assert f"STATUS {knn.KNN_ENOMEM} {knn.KNN_EINVAL} 0 0 True" in r.stdout, r.stdout
