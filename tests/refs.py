"""Independent numpy statements used to pin the oracle (test helpers only).

These are written from the mathematics, not from the oracle's C code:
exhaustive KNN under the (squared distance, index) order, and the set form of
the layer-by-layer stop rule.
"""
import numpy as np


def sqdist_f32(points: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Squared Euclidean distances in float32, summed in dimension order.

    Every numpy float32 operation rounds to nearest on its own, so no product is
    fused with the following addition.
    """
    acc = np.zeros(points.shape[0], np.float32)
    for j in range(points.shape[1]):
        t = np.float32(q[j]) - points[:, j]
        acc = acc + t * t
    return acc


def knn_exhaustive(points: np.ndarray, q: np.ndarray, k: int, subset=None):
    """k nearest under (dist2, index) ascending; -1 / +inf padding."""
    d2 = sqdist_f32(points, q)
    idx = np.arange(points.shape[0])
    if subset is not None:
        d2, idx = d2[subset], idx[subset]
    order = np.lexsort((idx, d2))[:k]
    ids = np.full(k, -1, np.int32)
    dd = np.full(k, np.inf, np.float32)
    ids[:len(order)] = idx[order]
    dd[:len(order)] = d2[order]
    return ids, dd


def set_form(points, pcells, q, c0, cmax, k):
    """Result of the layer walk restated on sets.

    T_L is the top-k of the points whose cell lies within Chebyshev distance L
    of the central cell c0.  The walk stops at the first layer L (from the
    first layer reaching the box of occupied cells) with |T_{L-1}| = k and
    T_L = T_{L-1}, or when cube(L) covers that box.  Returns (ids, dist2, L*).
    """
    cheb = np.abs(pcells - c0[None, :]).max(axis=1)
    lmin = int(np.max(np.maximum(0, np.maximum(-c0, c0 - cmax))))
    prev = None
    L = lmin
    while True:
        ids, dd = knn_exhaustive(points, q, k, subset=np.nonzero(cheb <= L)[0])
        covers = bool(np.all(c0 - L <= 0) and np.all(c0 + L >= cmax))
        if prev is not None and (prev >= 0).all() and np.array_equal(prev, ids):
            return ids, dd, L
        if covers:
            return ids, dd, L
        prev = ids
        L += 1


def vote(labels):
    """Majority label; ties go to the smallest label."""
    vals, counts = np.unique(np.asarray(labels), return_counts=True)
    return int(vals[np.argmax(counts)])  # np.unique sorts, argmax takes the first max
