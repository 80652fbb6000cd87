"""GHN oracle: plain, slow CPU statement of the grid-hashing KNN method.

Test infrastructure only.  The test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only code that imports this package; the product
path (the CUDA library and its binding) never does.  Nothing here is shared
with the CUDA library.
"""
from .oracle import (  # noqa: F401
    RULE_EXACT,
    RULE_NONE,
    RULE_PAPER,
    Grid,
    brute_force,
    build_library,
    count_cells,
    library,
    measure_cells,
    recall,
    shell_count,
)
