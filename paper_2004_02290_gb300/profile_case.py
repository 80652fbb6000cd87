"""One index build and one query launch of a named workload, for profilers.

  python -m paper_2004_02290_gb300.profile_case --config large_cls --m 50000
  python -m paper_2004_02290_gb300.profile_case --batched-problem 100 --width 0.11656

Keeps the capture small: the full training set of the workload (so the index
has its real shape) and a prefix of its queries.  Prints the phase times.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--config", default="large_cls")
    p.add_argument("--m", type=int, default=None, help="queries (a prefix of the workload's)")
    p.add_argument("--repeat", type=int, default=1)
    p.add_argument("--sorted", action="store_true", help="visit queries in cell order")
    p.add_argument("--batched-problem", type=int, default=None,
                   help="problem i of the 256-problem batched workload instead of --config")
    p.add_argument("--width", type=float, default=None, help="cell width (with --batched-problem)")
    args = p.parse_args(argv)

    import torch

    import __graft_entry__
    from paper_2004_02290_gb300 import knn
    from paper_2004_02290_gb300 import workloads as wl

    __graft_entry__.build()
    if args.batched_problem is not None:
        if args.width is None:
            raise SystemExit("--batched-problem needs --width")
        w = wl.gen_batched(256, seed=3)[args.batched_problem]
        w.w = float(args.width)
        if args.m is not None:
            w.queries = w.queries[: args.m]
    else:
        w = wl.make(args.config, m=args.m)
    dev = torch.device("cuda:0")
    pts = torch.from_numpy(w.points).to(dev)
    lab = torch.from_numpy(w.labels).to(dev)
    q = torch.from_numpy(w.queries).to(dev)
    flags = knn.KNN_QUERY_CHECKED | (knn.KNN_QUERY_SORTED if args.sorted else 0)
    knn.knn_timing_enable(True)
    idx = knn.knn_build(pts, lab, w.w, w.table)
    print("build:", knn.knn_timing_read())
    for _ in range(args.repeat):
        idx.query(q, w.k, w.mode, flags=flags)
        print("query:", knn.knn_timing_read())
    torch.cuda.synchronize()
    inf = idx.info()
    print(f"{w.name}: n={w.n} m={w.m} d={w.d} k={w.k} cells={inf.num_cells} "
          f"table={'dense' if inf.table == 1 else 'hash'} slots={inf.table_slots}")
    idx.free()


if __name__ == "__main__":
    main()
