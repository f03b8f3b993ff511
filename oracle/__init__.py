"""Plain FP64 CPU oracle of the staggered-grid Stokes system, its multigrid pieces and the outer
accelerators (GCR, Anderson).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product library neither imports nor links it.
"""
from . import stokes, multigrid, accelerators  # noqa: F401
