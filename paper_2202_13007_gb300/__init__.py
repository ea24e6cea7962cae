"""GB300 (sm_103a) implementation of the blaz compressed-matrix method
("Compressed Matrix Computations", arXiv 2202.13007).

The CUDA kernels and the C ABI live in ``csrc/`` and ``include/blaz.h``;
``blaz`` is the thin Python binding.
"""
from . import blaz  # noqa: F401
from .blaz import CMat, BlazError  # noqa: F401
