"""Autotuner for each index of a problem set: cell width and threads per query.

The paper measures cells from the data (Sec. III.A); the library takes the
width from the caller.  For a problem set, the tuner picks each index's
settings by measurement on the GPU:
  - cell width: starting from a guess, it walks a grid of widths (half powers
    of two) downhill, building the index and timing a sample of the queries
    at each, and keeps the width of the least estimated time (build + sampled
    query time scaled to all queries);
  - threads per query for heavy queries: at that width, it times the sample
    with the library's default deferral to the cooperative kernel (a block
    of 512 threads for a query whose layers or row batches are large), with
    no deferral by candidate count, and with no deferral at all (every query
    on one warp of 32 threads), and keeps the fastest
    (knn_index_set_deferral / knn_batch_set_deferral).  In a batch the
    problems of one kernel group share their launches, so the batch-level
    pass (refine_batch_deferral) then times each group's deferral inside the
    batched query itself.
The warp kernel's own tile (32 rows a batch, 32 candidates a chunk, the
resident blocks per SM) is fixed by the design and its occupancy sweep.

Every candidate runs through the same library calls as a normal query, so
the chosen width is an input like any other: the oracle takes it unchanged.
The deferral changes which kernel walks a query, never its result.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import knn


# Deferral settings the tuner tries (heavy_rows, heavy_cands): the library's
# default, no deferral by candidate count, no deferral.
DEFERRALS = [(0, 0), (0, -1), (-1, -1)]


@dataclasses.dataclass
class Choice:
    width: float
    est_ms: float
    tried: list  # (width, est_ms)
    deferral: tuple = (0, 0)  # (heavy_rows, heavy_cands) of knn_index_set_deferral
    deferral_ms: list = dataclasses.field(default_factory=list)  # sample ms per DEFERRALS entry


def start_width(points, k: int) -> float:
    """A first guess: cells holding about max(2, k/2) points if the data filled its box.

    points: n x d numpy array or torch tensor.
    """
    n, d = int(points.shape[0]), int(points.shape[1])
    if hasattr(points, "amin"):  # torch tensor: reduce on its device
        lo = points.amin(dim=0).double().cpu().numpy()
        hi = points.amax(dim=0).double().cpu().numpy()
    else:
        lo = points.min(axis=0).astype(np.float64)
        hi = points.max(axis=0).astype(np.float64)
    span = np.maximum(hi - lo, 1e-12)
    vol = float(np.prod(span))
    occ = max(2.0, k / 2.0)
    return float(np.float32((vol * occ / n) ** (1.0 / d)))


def _estimate(pts, lab, q, k, mode, m, s, w, stream):
    """Build + sampled query time (ms) at width w, query time scaled to m; None if unbuildable."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    try:
        ev[0].record(stream)
        idx = knn.knn_build(pts, lab, w)
        ev[1].record(stream)
        idx.query(q, k, mode if lab is not None else knn.KNN_NONE)
        ev[2].record(stream)
        ev[2].synchronize()
        idx.free()
    except knn.KnnError:
        return None  # a width the index cannot hold (grid too fine)
    return ev[0].elapsed_time(ev[1]) + ev[1].elapsed_time(ev[2]) * (m / s)


def tune_width(points, labels, queries, k: int, mode: int, step: float = 0.5,
               max_steps: int = 10, sample: int = 4096, dev=None) -> Choice:
    """Width of least estimated build + query time for one problem (GPU).

    Walks downhill on a grid of widths w0 * 2^(step * i) from the starting
    guess w0, one step at a time, until the cost rises (at most max_steps
    steps each way).
    """
    import torch

    dev = dev or torch.device("cuda:0")

    def on_dev(a):
        if a is None:
            return None
        if isinstance(a, torch.Tensor):
            return a.to(dev).contiguous()
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    pts = on_dev(points)
    if pts.dtype != torch.float32:
        raise ValueError("points must be float32")
    w0 = start_width(pts, k)
    lab = on_dev(labels)
    m = int(queries.shape[0])
    s = min(sample, m)
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(m, size=s, replace=False)) if s < m else np.arange(m)
    if isinstance(queries, torch.Tensor):
        q = queries.to(dev)[torch.from_numpy(pick).to(dev)].contiguous()
    else:
        q = on_dev(np.ascontiguousarray(queries[pick], np.float32))
    stream = torch.cuda.current_stream(dev)
    cache = {}

    def cost(i):
        if i not in cache:
            w = float(np.float32(w0 * 2.0 ** (step * i)))
            cache[i] = (w, _estimate(pts, lab, q, k, mode, m, s, w, stream))
        return cache[i][1]

    i = 0
    c0 = cost(0)
    if c0 is None:
        i, c0 = 1, cost(1)
    for direction in (-1, 1):
        j = i
        for _ in range(max_steps):
            c = cost(j + direction)
            if c is None or c0 is None or c >= c0:
                break
            j += direction
            c0 = c
        i = j
    tried = sorted((w, c) for w, c in cache.values() if c is not None)
    if not tried:
        raise RuntimeError("no candidate width could be built")
    best = min(tried, key=lambda t: t[1])
    deferral, dms = _tune_deferral(pts, lab, q, k, mode, best[0], stream)
    return Choice(width=best[0], est_ms=best[1], tried=tried, deferral=deferral,
                  deferral_ms=dms)


def _tune_deferral(pts, lab, q, k, mode, w, stream, reps: int = 3):
    """The fastest deferral setting on the sample (least of `reps` timings each)."""
    import torch

    idx = knn.knn_build(pts, lab, w)
    md = mode if lab is not None else knn.KNN_NONE
    times = []
    for rows, cands in DEFERRALS:
        idx.set_deferral(rows, cands)
        best = None
        for _ in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            idx.query(q, k, md)
            ev[1].record(stream)
            ev[1].synchronize()
            t = ev[0].elapsed_time(ev[1])
            best = t if best is None else min(best, t)
        times.append(best)
    idx.free()
    i = min(range(len(DEFERRALS)), key=lambda j: times[j])
    return DEFERRALS[i], times


def tune_batch(problems, dev=None):
    """Settings for every problem; returns (widths, seconds spent, choices)
    (each choice also carries the problem's deferral setting)."""
    t0 = time.perf_counter()
    choices = [tune_width(p.points, p.labels, p.queries, p.k, p.mode, dev=dev) for p in problems]
    return [c.width for c in choices], time.perf_counter() - t0, choices


def refine_batch_deferral(problems, widths, defer, dev=None, reps: int = 3):
    """Deferral settings per kernel group, measured in the batched query.

    A group is the problems that share one launch (dimension, k up to 32 or
    more, table kind).  For each group the batch is queried with the group's
    problems on their own per-problem settings (`defer`), all on the
    library's default and all on no deferral; the group's phase times (its
    warp and cooperative launches, from the library's phase events) decide,
    least of `reps` timings each.  Other groups keep their settings while one
    is tried.  The library's phase timing is left off.  Returns (settings per
    problem, seconds spent, {group phase: chosen option}).
    """
    import torch

    t0 = time.perf_counter()
    dev = dev or torch.device("cuda", torch.cuda.current_device())
    pts = [torch.from_numpy(np.ascontiguousarray(p.points)).to(dev) for p in problems]
    lab = [torch.from_numpy(np.ascontiguousarray(p.labels)).to(dev) for p in problems]
    qs = [torch.from_numpy(np.ascontiguousarray(p.queries)).to(dev) for p in problems]
    ks = [p.k for p in problems]
    modes = [p.mode for p in problems]
    b = knn.knn_batch_build(pts, lab, widths)
    groups = {}
    for i, p in enumerate(problems):
        dense = b.info(i).table == knn.KNN_TABLE_DENSE
        g = f"query.d{p.d}.{'k64' if p.k > 32 else 'k32'}.{'dense' if dense else 'hash'}"
        groups.setdefault(g, []).append(i)
    cur = [tuple(x) for x in defer]

    def group_ms(g, settings):
        for i in groups[g]:
            b.set_deferral(i, *settings[i])
        best = None
        for _ in range(reps):
            while knn.knn_timing_read():
                pass
            b.query(qs, ks, modes)
            torch.cuda.synchronize(dev)
            t = sum(ms for n, ms in knn.knn_timing_read() if n == g or n.startswith(g + "."))
            best = t if best is None else min(best, t)
        return best

    knn.knn_timing_enable(True)
    chosen = {}
    try:
        for g, members in groups.items():
            options = {"per problem": list(cur)}
            for name, x in (("default", (0, 0)), ("none", (-1, -1))):
                opt = list(cur)
                for i in members:
                    opt[i] = x
                options[name] = opt
            times = {name: group_ms(g, opt) for name, opt in options.items()}
            name = min(times, key=times.get)
            cur = options[name]
            for i in members:
                b.set_deferral(i, *cur[i])
            chosen[g] = name
    finally:
        knn.knn_timing_enable(False)
        b.free()
    return cur, time.perf_counter() - t0, chosen
