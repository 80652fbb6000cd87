"""knn_query_noalloc, the query entry point that allocates nothing.

It serves callers that cannot allocate device memory while they query (their
own allocator already holds the GPU, or their loop must not pay an
allocation's latency).  Its results must equal knn_query's on the same index,
on two calls in a row that share the library's fixed scratch array.  This file
is collected last, so a failure here stops a -x run only after every other
test has run.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2004_02290_gb300 import knn
from paper_2004_02290_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MEAN_RTOL = 1e-6
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _noalloc(idx, q, k, mode):
    m = q.shape[0]
    ids = torch.full((m, k), -7, dtype=torch.int32, device="cuda")
    d2 = torch.full((m, k), -7.0, dtype=torch.float32, device="cuda")
    pred = torch.full((m,), -7, dtype=torch.int32 if mode == knn.KNN_VOTE else torch.float32,
                      device="cuda")
    lib = knn.library()
    rc = lib.knn_query_noalloc(idx.handle, q.data_ptr(), m, k, mode, ids.data_ptr(),
                               d2.data_ptr(), pred.data_ptr(), knn.KNN_QUERY_CHECKED,
                               torch.cuda.current_stream().cuda_stream)
    assert rc == knn.KNN_OK, lib.knn_last_error()
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d2.cpu().numpy(), pred.cpu().numpy()


def _same(a, b, mode):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    if mode == knn.KNN_VOTE:
        assert np.array_equal(a[2], b[2])
    else:
        rel = np.abs(a[2].astype(np.float64) - b[2]) / np.maximum(np.abs(b[2]), 1e-30)
        assert rel.max() <= MEAN_RTOL


def test_noalloc_matches_knn_query_twice():
    # clustered data: some queries go through the cooperative kernel, whose
    # list of deferred queries also lives in the fixed scratch array
    w = wl.make("skewed_reg", n=200_000, m=6000, w=0.02)
    idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w)
    q1 = _dev(w.queries)
    q2 = _dev(w.queries[::-1][:2500])
    for q in (q1, q2):  # two calls in a row, the second with fewer queries
        ids, d2, pred = idx.query(q, w.k, w.mode, flags=knn.KNN_QUERY_CHECKED)
        ref = (ids.cpu().numpy(), d2.cpu().numpy(), pred.cpu().numpy())
        _same(_noalloc(idx, q, w.k, w.mode), ref, w.mode)
    idx.free()


def test_noalloc_vote_hash_table():
    w = wl.make("large_cls", n=60_000, m=3000, w=0.03)
    idx = knn.knn_build(_dev(w.points), _dev(w.labels), w.w, knn.KNN_TABLE_HASH)
    q = _dev(w.queries)
    ids, d2, pred = idx.query(q, w.k, w.mode, flags=knn.KNN_QUERY_CHECKED)
    ref = (ids.cpu().numpy(), d2.cpu().numpy(), pred.cpu().numpy())
    for _ in range(2):
        _same(_noalloc(idx, q, w.k, w.mode), ref, w.mode)
    idx.free()


def test_noalloc_rejects_too_many_queries_and_host_buffers():
    x, lab, q = wl.uniform(1000, 8, 2, seed=3)
    idx = knn.knn_build(_dev(x), _dev(lab), 0.05)
    lib = knn.library()
    ids = torch.empty((8, 3), dtype=torch.int32, device="cuda")
    qd = _dev(q)
    rc = lib.knn_query_noalloc(idx.handle, qd.data_ptr(), (1 << 20) + 1, 3, -1, ids.data_ptr(),
                               None, None, 0, None)
    assert rc == knn.KNN_EINVAL
    assert b"1048576" in lib.knn_last_error()
    host_ids = np.zeros((8, 3), np.int32)
    rc = lib.knn_query_noalloc(idx.handle, qd.data_ptr(), 8, 3, -1, host_ids.ctypes.data, None,
                               None, 0, None)
    assert rc == knn.KNN_EINVAL
    assert b"device memory" in lib.knn_last_error()
    idx.free()


_ALL_DEFERRED = r"""
import numpy as np, torch
from paper_2004_02290_gb300 import knn, workloads as wl
def dev(a): return torch.from_numpy(np.ascontiguousarray(a)).cuda()
lib = knn.library()
w = wl.make("skewed_reg", n=50_000, m=3000, w=0.03)
idx = knn.knn_build(dev(w.points), dev(w.labels), w.w)
bad = 0
for q in (dev(w.queries), dev(w.queries[::-1][:1200])):
    ids, d2, pred = idx.query(q, w.k, w.mode, flags=knn.KNN_QUERY_CHECKED)
    m = q.shape[0]
    ids2 = torch.full((m, w.k), -7, dtype=torch.int32, device="cuda")
    d22 = torch.full((m, w.k), -7.0, dtype=torch.float32, device="cuda")
    pred2 = torch.full((m,), -7.0, dtype=torch.float32, device="cuda")
    rc = lib.knn_query_noalloc(idx.handle, q.data_ptr(), m, w.k, w.mode, ids2.data_ptr(),
                               d22.data_ptr(), pred2.data_ptr(), knn.KNN_QUERY_CHECKED,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    bad += rc != 0
    bad += not torch.equal(ids, ids2)
    bad += not torch.equal(d2.view(torch.int32), d22.view(torch.int32))
    bad += not torch.equal(pred.view(torch.int32), pred2.view(torch.int32))
idx.free()
print("BAD", bad)
"""


def test_noalloc_every_query_deferred():
    """Every query handed to the cooperative kernel, whose list of deferred
    queries is in the fixed array: both calls, the second shorter, must still
    equal knn_query bit for bit."""
    env = dict(os.environ, GHN_HEAVY_ROWS="2", GHN_HEAVY_CANDS="8")
    r = subprocess.run([sys.executable, "-c", _ALL_DEFERRED], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "BAD 0" in r.stdout, r.stdout
