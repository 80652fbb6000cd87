"""Cell-width search: pick the grid width w for a target mean occupancy.

Test and workload infrastructure.  The paper measures cells per dimension from
the data (Sec. III.A); the library takes one scalar width from the caller, so
the workloads fix w once by a geometric bisection on the number of occupied
cells counted with the oracle's own key function (Eq. 1).

Run ``python -m oracle.cell_width`` to print the full-size widths stored in
``paper_2004_02290_gb300/workloads.py`` (this takes a few minutes for the
20-million-point workload).
"""
from __future__ import annotations

import math
import sys

import numpy as np

from .oracle import count_cells


def search_width(points: np.ndarray, occupancy: float, iters: int = 24,
                 lo: float = 1e-5, hi: float = 4.0) -> float:
    """Float32 width whose mean occupancy n / #occupied-cells is closest to `occupancy`."""
    n = points.shape[0]
    best_w, best_err = None, math.inf
    a, b = math.log(lo), math.log(hi)
    for _ in range(iters):
        mid = 0.5 * (a + b)
        w = float(np.float32(math.exp(mid)))
        occ = n / count_cells(points, w)
        err = abs(math.log(occ / occupancy))
        if err < best_err:
            best_w, best_err = w, err
        if occ < occupancy:
            a = mid
        else:
            b = mid
    return best_w


def main(argv):
    sys.path.insert(0, ".")
    from paper_2004_02290_gb300 import workloads as wl

    names = argv[1:] or list(wl.SPECS)
    for name in names:
        spec = wl.SPECS[name]
        x, _, _ = wl._GEN[name](n=spec["n"], m=1, seed=spec["seed"])
        w = search_width(x, spec["occupancy"])
        occ = x.shape[0] / count_cells(x, w)
        bits = np.float32(w).view(np.uint32)
        print(f"{name}: w={w!r} (float32 bits 0x{bits:08x}), mean occupancy {occ:.3f}",
              flush=True)


if __name__ == "__main__":
    main(sys.argv)
