"""Seeded synthetic workloads shaped like the paper's experiments.

The paper evaluates on PCA-reduced public datasets (Sec. IV, Table I) that are
not available here.  These generators stand in for them.  Each draws training
points, 32-bit outputs and queries from a seeded numpy PCG64 stream in float64
and rounds the draws to float32.  This module holds no arithmetic of the method
itself (no cell keys, no distances); it only draws random numbers, so the oracle
and the CUDA library can both be fed from it.

Workloads (the paper's setting is KNN classification and regression, Sec. I):

  tiny        d=2, n=10,000, 4 equal-weight Gaussian blobs (sigma 0.08, centres
              uniform in [0,1]^2, clipped to [0,1]), int32 label = blob id;
              1,000 queries from the same mixture; k=5, vote; seed 0.
  large_cls   d=4, n=2,000,000, 16 equal-weight clusters (sigma 0.04, centres
              uniform in [0,1]^4, unclipped), label = cluster id with 5% of the
              points relabelled uniformly to one of the other 15; 200,000
              queries from the mixture; k=10, vote; open-addressing hash table.
  skewed_reg  d=3, n=20,000,000, 70% from 8 tight clusters (sigma 0.01, centres
              uniform in [0,1]^3), 30% uniform in [0,1]^3; target
              y = sin(6 x0) + x1 x2 + N(0, 0.05^2) in float64, rounded to float32;
              1,000,000 queries uniform in [0,1]^3; k=16, mean; seed 2.

Cell widths are fixed float32 constants per workload.  Each was chosen once,
by a geometric bisection on the number of occupied cells of the full-size
training set, for a mean occupancy of about 8 (tiny, skewed_reg) or 4
(large_cls) points per occupied cell.  The search script sits with the oracle
and prints these values.
"""
from __future__ import annotations

import dataclasses

import numpy as np

VOTE = 0
MEAN = 1

TABLE_AUTO = 0
TABLE_DENSE = 1
TABLE_HASH = 2


@dataclasses.dataclass
class Workload:
    name: str
    points: np.ndarray    # n x d float32, row-major
    labels: np.ndarray    # n int32 (vote) or float32 (mean)
    queries: np.ndarray   # m x d float32
    k: int
    mode: int             # VOTE or MEAN
    w: float              # cell width (float32 value)
    table: int            # TABLE_AUTO / TABLE_DENSE / TABLE_HASH
    seed: int

    @property
    def n(self) -> int:
        return self.points.shape[0]

    @property
    def d(self) -> int:
        return self.points.shape[1]

    @property
    def m(self) -> int:
        return self.queries.shape[0]


def _f32_bits(b: int) -> float:
    return float(np.array([b], np.uint32).view(np.float32)[0])


# Full-size cell widths as float32 bit patterns (see the module docstring):
# tiny 0.018221075 (mean occupancy 8.006), large_cls 0.013427479 (4.000),
# skewed_reg 0.0070754485 (8.000).
WIDTHS = {
    "tiny": _f32_bits(0x3C95445D),
    "large_cls": _f32_bits(0x3C5BFEEE),
    "skewed_reg": _f32_bits(0x3BE7D92A),
}

SPECS = {
    "tiny": dict(d=2, n=10_000, m=1_000, k=5, mode=VOTE, seed=0, table=TABLE_AUTO,
                 occupancy=8.0),
    "large_cls": dict(d=4, n=2_000_000, m=200_000, k=10, mode=VOTE, seed=1, table=TABLE_HASH,
                      occupancy=4.0),
    "skewed_reg": dict(d=3, n=20_000_000, m=1_000_000, k=16, mode=MEAN, seed=2,
                       table=TABLE_AUTO, occupancy=8.0),
}


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def gen_tiny(n=10_000, m=1_000, seed=0):
    rng = np.random.default_rng(seed)
    centres = rng.random((4, 2))

    def draw(count):
        comp = rng.integers(0, 4, size=count)
        x = np.clip(centres[comp] + 0.08 * rng.standard_normal((count, 2)), 0.0, 1.0)
        return x, comp

    x, comp = draw(n)
    q, _ = draw(m)
    return _f32(x), comp.astype(np.int32), _f32(q)


def gen_large_cls(n=2_000_000, m=200_000, seed=1):
    rng = np.random.default_rng(seed)
    centres = rng.random((16, 4))

    def draw(count):
        comp = rng.integers(0, 16, size=count)
        return centres[comp] + 0.04 * rng.standard_normal((count, 4)), comp

    x, comp = draw(n)
    lab = comp.copy()
    flip = rng.random(n) < 0.05
    # relabel uniformly to one of the other 15 clusters
    shift = rng.integers(1, 16, size=n)
    lab[flip] = (comp[flip] + shift[flip]) % 16
    q, _ = draw(m)
    return _f32(x), lab.astype(np.int32), _f32(q)


def gen_skewed_reg(n=20_000_000, m=1_000_000, seed=2):
    rng = np.random.default_rng(seed)
    centres = rng.random((8, 3))
    n_clu = int(round(0.7 * n))
    comp = rng.integers(0, 8, size=n_clu)
    x = np.empty((n, 3), np.float64)
    x[:n_clu] = centres[comp] + 0.01 * rng.standard_normal((n_clu, 3))
    x[n_clu:] = rng.random((n - n_clu, 3))
    # shuffle so that training indices carry no cluster structure
    perm = rng.permutation(n)
    x = x[perm]
    xf = _f32(x)
    xd = xf.astype(np.float64)
    y = np.sin(6.0 * xd[:, 0]) + xd[:, 1] * xd[:, 2] + 0.05 * rng.standard_normal(n)
    q = rng.random((m, 3))
    return xf, y.astype(np.float32), _f32(q)


_GEN = {"tiny": gen_tiny, "large_cls": gen_large_cls, "skewed_reg": gen_skewed_reg}


def make(name: str, n: int | None = None, m: int | None = None, w: float | None = None,
         seed: int | None = None) -> Workload:
    """The named workload at full size, or resized (n, m) with a caller-given width.

    A resized workload keeps the distribution; its width must be given (the
    stored widths belong to the full-size training sets).
    """
    spec = SPECS[name]
    n_ = spec["n"] if n is None else int(n)
    m_ = spec["m"] if m is None else int(m)
    seed_ = spec["seed"] if seed is None else int(seed)
    if w is None:
        if n_ != spec["n"] or seed_ != spec["seed"]:
            raise ValueError("a resized workload needs an explicit cell width")
        w = WIDTHS[name]
        if w is None:
            raise ValueError(f"no stored cell width for {name}")
    x, lab, q = _GEN[name](n=n_, m=m_, seed=seed_)
    return Workload(name=name, points=x, labels=lab, queries=q, k=spec["k"], mode=spec["mode"],
                    w=float(np.float32(w)), table=spec["table"], seed=seed_)


def uniform(n, m, d, seed, lo=0.0, hi=1.0, classes=4):
    """Uniform points/queries in [lo, hi)^d with random int32 labels (parity cases)."""
    rng = np.random.default_rng(seed)
    x = lo + (hi - lo) * rng.random((n, d))
    q = lo + (hi - lo) * rng.random((m, d))
    lab = rng.integers(0, classes, size=n).astype(np.int32)
    return _f32(x), lab, _f32(q)


def lattice(side, d, m, seed):
    """Integer lattice points (many exact distance ties) and integer-ish queries."""
    rng = np.random.default_rng(seed)
    axes = [np.arange(side, dtype=np.float64)] * d
    x = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, d)
    x = x[rng.permutation(x.shape[0])]
    q = np.round(rng.random((m, d)) * (side - 1) * 2) / 2.0
    lab = rng.integers(0, 3, size=x.shape[0]).astype(np.int32)
    return _f32(x), lab, _f32(q)


def regression_targets(points, seed):
    """Smooth float32 targets with noise, for mean-mode parity cases."""
    rng = np.random.default_rng(seed)
    p = points.astype(np.float64)
    y = np.sin(3.0 * p[:, 0]) + 0.5 * p.sum(axis=1) + 0.01 * rng.standard_normal(p.shape[0])
    return y.astype(np.float32)


def gen_batched(count=256, seed=3, n_lo=1_000, n_hi=2_000_000, dims=(2, 3, 4, 6),
                ks=(1, 5, 15, 32)):
    """Many independent problems of uneven size, for the batched form.

    Per problem: n log-uniform in [n_lo, n_hi], d uniform in `dims`, k uniform
    in `ks`, m = n // 10 queries (at least 1) from the same mixture; points
    from a Gaussian mixture with 4..32 clusters (centres uniform in [0,1]^d,
    sigma uniform in [0.02, 0.1]).  Even problems are classification (label =
    cluster), odd ones regression (a smooth target plus noise).  Cell widths
    are left unset (w = nan): the autotuner chooses them.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        d = int(rng.choice(dims))
        k = int(rng.choice(ks))
        m = max(1, n // 10)
        ncl = int(rng.integers(4, 33))
        sigma = float(rng.uniform(0.02, 0.1))
        centres = rng.random((ncl, d))
        comp = rng.integers(0, ncl, size=n)
        x = _f32(centres[comp] + sigma * rng.standard_normal((n, d)))
        qc = rng.integers(0, ncl, size=m)
        q = _f32(centres[qc] + sigma * rng.standard_normal((m, d)))
        if i % 2 == 0:
            mode, lab = VOTE, comp.astype(np.int32)
        else:
            xd = x.astype(np.float64)
            y = np.sin(3.0 * xd[:, 0]) + 0.5 * xd.sum(axis=1) + 0.05 * rng.standard_normal(n)
            mode, lab = MEAN, y.astype(np.float32)
        out.append(Workload(name=f"batched[{i}]", points=x, labels=lab, queries=q, k=k,
                            mode=mode, w=float("nan"), table=TABLE_AUTO, seed=seed))
    return out


# ---- the serving workload: resident indexes and a Poisson request stream ----

@dataclasses.dataclass
class ServeIndex:
    """One index of the serving workload: a Gaussian mixture, drawn on demand."""
    n: int
    d: int
    mode: int             # VOTE (label = cluster) or MEAN (smooth target + noise)
    centres: np.ndarray   # ncl x d, float64
    sigma: float
    seed: int


@dataclasses.dataclass
class ServeEvent:
    t: float              # arrival, seconds from the start
    kind: str             # "query" or "build"
    index: int = -1       # query: position in the resident list
    queries: np.ndarray | None = None
    k: int = 0
    mode: int = -1
    spec: ServeIndex | None = None  # build: the new index


def _serve_index(rng, n, d, seed):
    ncl = int(rng.integers(4, 33))
    return ServeIndex(n=n, d=d, mode=VOTE if seed % 2 == 0 else MEAN,
                      centres=rng.random((ncl, d)), sigma=float(rng.uniform(0.02, 0.1)),
                      seed=seed)


def gen_serving_indexes(count=64, seed=5, n_lo=10_000, n_hi=50_000_000, dims=(2, 3, 4, 5, 6),
                        cap_bytes=60 << 30, bytes_per_point=72):
    """Resident indexes of the serving workload.

    n log-uniform in [n_lo, n_hi], d uniform in `dims`, 4..32 clusters with
    centres uniform in [0,1]^d and one sigma uniform in [0.02, 0.1]; even
    positions classify, odd ones regress.  When the indexes would hold more
    than cap_bytes (at bytes_per_point per point, an over-estimate of the
    resident size), every n is scaled down by the same factor.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        d = int(rng.choice(dims))
        out.append(_serve_index(rng, n, d, seed * 1000 + i))
    total = sum(ix.n for ix in out) * bytes_per_point
    if total > cap_bytes:
        f = cap_bytes / total
        for ix in out:
            ix.n = max(n_lo, int(ix.n * f))
    return out


def serving_points(ix: ServeIndex, device):
    """(points n x d float32, labels) of an index, drawn on `device` from a seeded torch stream."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(ix.seed)
    c = torch.from_numpy(ix.centres).to(device=device, dtype=torch.float64)
    comp = torch.randint(0, c.shape[0], (ix.n,), generator=g, device=device)
    x = c[comp] + ix.sigma * torch.randn((ix.n, ix.d), generator=g, device=device,
                                         dtype=torch.float64)
    pts = x.to(torch.float32).contiguous()
    if ix.mode == VOTE:
        lab = comp.to(torch.int32)
    else:
        xd = pts.to(torch.float64)
        y = torch.sin(3.0 * xd[:, 0]) + 0.5 * xd.sum(dim=1) + 0.05 * torch.randn(
            ix.n, generator=g, device=device, dtype=torch.float64)
        lab = y.to(torch.float32)
    del x, comp
    return pts, lab.contiguous()


def serving_queries(ix: ServeIndex, m: int, rng) -> np.ndarray:
    """m queries from an index's mixture (host, float32)."""
    comp = rng.integers(0, ix.centres.shape[0], size=m)
    return _f32(ix.centres[comp] + ix.sigma * rng.standard_normal((m, ix.d)))


def gen_serving_requests(indexes, rate=2000.0, duration=10.0, seed=6, m_lo=1, m_hi=4096,
                         ks=(5, 16), build_rate=4.0, build_n=(10_000, 5_000_000),
                         dims=(2, 3, 4, 5, 6)):
    """Poisson arrivals over `duration` seconds.

    Query requests arrive at `rate` per second; each names a resident index
    uniformly, has m log-uniform in [m_lo, m_hi] queries from that index's
    mixture and k uniform in `ks`, with the index's own head.  Build requests
    arrive at `build_rate` per second, each for a new index with n
    log-uniform in `build_n`.
    """
    rng = np.random.default_rng(seed)
    events = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        i = int(rng.integers(0, len(indexes)))
        ix = indexes[i]
        m = int(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi + 1))))
        m = min(max(m, m_lo), m_hi)
        events.append(ServeEvent(t=t, kind="query", index=i, queries=serving_queries(ix, m, rng),
                                 k=int(rng.choice(ks)), mode=ix.mode))
    t = 0.0
    j = 0
    while build_rate > 0:
        t += rng.exponential(1.0 / build_rate)
        if t >= duration:
            break
        n = int(round(np.exp(rng.uniform(np.log(build_n[0]), np.log(build_n[1])))))
        events.append(ServeEvent(t=t, kind="build",
                                 spec=_serve_index(rng, n, int(rng.choice(dims)),
                                                   seed * 100000 + j)))
        j += 1
    events.sort(key=lambda e: e.t)
    return events
