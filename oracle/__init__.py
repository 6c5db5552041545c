"""FP64 CPU oracle of the lock-exchange LBM step (arXiv 2112.08479).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product library never
imports, links or runs anything here, and this package imports nothing from
the product library.
"""
from .oracle import *  # noqa: F401,F403
