"""CPU FP64 oracle for the Hierarchical Approximate POD (arXiv 1607.05210).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product path never does.  It
shares no code with the CUDA library (``paper_1607_05210_gb300``) and never
imports it.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute-force SVD on tiny inputs, prescribed spectra, the advection-diffusion
closed form, the theorems of Sec. 3.3 and hand-derived tolerance values).
"""
from .core import (  # noqa: F401
    gram,
    svd,
    pod,
    tail_sums,
    tree_levels,
    accumulated_counts,
    tolerances,
    hapod,
    projection_error,
)
