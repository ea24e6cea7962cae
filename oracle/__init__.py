"""CPU oracle of the blaz compressed-matrix method (arXiv 2202.13007).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product path (the CUDA
library and its Python binding) never imports, links or calls anything here,
and this package imports nothing from the product.

The arithmetic lives in ``blaz_oracle.c`` (plain single-threaded C compiled
without FMA contraction); ``oracle.py`` marshals numpy arrays into it.
"""
from .oracle import *  # noqa: F401,F403
