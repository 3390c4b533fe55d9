"""hapod_gram_noalloc, the Gram entry point for callers that cannot allocate device
memory while running (their own allocator holds the GPU's memory, or allocation
latency is not acceptable), must give the same Gram matrix as hapod_gram.

The file sorts last so that a run stopping at the first failure has run every
other test before it.  It also passes on its own in a fresh process.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from tests.helpers import to_dev

pytestmark = pytest.mark.gpu


def _gram_tol(X, n):
    d = np.sqrt(np.sum(X * X, axis=0))
    return 1e-13 * math.sqrt(n) * np.outer(d, d)  # tolerance of the FP64 Gram parity tests


def test_noalloc_gram_matches_hapod_gram_twice(cuda_ok):
    from paper_1607_05210_gb300 import hapod as H

    rng = np.random.default_rng(20260101)
    cases = [(100_000, 150, 100_003), (40_000, 70, 40_000)]  # second call reuses the scratch of the first
    for n, m, ld in cases:
        X = rng.standard_normal((n, m)) * (1.0 + np.arange(m)) / m
        Xd = to_dev(X, ld=ld)
        G = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")
        st = H._lib.hapod_gram_noalloc(n, m, ctypes.c_void_p(Xd.data_ptr()), ld, ctypes.c_void_p(G.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == H.HAPOD_OK, H.hapod_last_error()
        ref = H.hapod_gram(Xd, H.HAPOD_FP64)
        torch.cuda.synchronize()
        Gh, Rh = G.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(Gh))
        assert np.all(np.abs(Gh - Rh) <= _gram_tol(X, n))


def test_noalloc_gram_rejects_too_wide(cuda_ok):
    from paper_1607_05210_gb300 import hapod as H

    X = to_dev(np.ones((1, 2900)))
    G = torch.empty((2900, 2900), dtype=torch.float64, device="cuda")
    st = H._lib.hapod_gram_noalloc(1, 2900, ctypes.c_void_p(X.data_ptr()), 1, ctypes.c_void_p(G.data_ptr()), None)
    assert st == H.HAPOD_ERR_INVALID
    assert "2816" in H.hapod_last_error()
