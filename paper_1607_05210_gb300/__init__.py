"""GB300-native Hierarchical Approximate POD (arXiv 1607.05210) hot path.

The compute path lives in the CUDA library ``_lib/libhapod.so`` (C ABI declared in
``include/hapod.h``); :mod:`paper_1607_05210_gb300.hapod` is the thin ctypes binding.
:mod:`paper_1607_05210_gb300.synth` holds the seeded input generators shared by the
tests and the benchmark.  Importing the package itself loads nothing; importing
``hapod`` loads the library and fails loudly if it has not been built.
"""
__all__ = ["hapod", "synth"]
