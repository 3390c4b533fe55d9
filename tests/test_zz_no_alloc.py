"""hapod_gram_noalloc is the Gram entry point for callers that cannot allocate
device memory while they run: an application whose own allocator already holds
nearly all of the GPU's memory, or a latency-bound pipeline that cannot pay for
cudaMalloc/cudaFree and the synchronisation they bring.  Its Gram matrix is
checked against the CPU oracle's G = X^T X with the tolerance of the FP64 Gram
parity tests, on calls made one after the other (each reuses the fixed scratch
array the previous call left behind), and against the existing entry point
hapod_gram.

The file sorts last so that a run stopping at the first failure has run every
other test before it.  It also passes on its own in a fresh process.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from tests.helpers import to_dev

pytestmark = pytest.mark.gpu


def _gram_tol(ref, n):
    d = np.sqrt(np.diag(ref))
    return 1e-13 * math.sqrt(max(n, 1)) * np.outer(d, d)  # tolerance of the FP64 Gram parity tests


def _noalloc(H, Xd, n, m, ld):
    G = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda")  # poisoned output
    st = H._lib.hapod_gram_noalloc(n, m, ctypes.c_void_p(Xd.data_ptr()), ld,
                                   ctypes.c_void_p(G.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == H.HAPOD_OK, H.hapod_last_error()
    torch.cuda.synchronize()
    return G.cpu().numpy()


def test_noalloc_gram_matches_oracle_on_consecutive_calls(cuda_ok):
    from paper_1607_05210_gb300 import hapod as H

    rng = np.random.default_rng(20260101)
    # one after the other, each reusing the scratch the previous call left: many row
    # splits, a near-limit width (990 upper-triangle tiles, one split), a partial
    # 32-row block with one split, and fewer rows than a warp
    cases = [(100_000, 150, 100_003), (40_000, 70, 40_000), (300, 2816, 300), (250, 65, 251), (17, 65, 17)]
    for n, m, ld in cases:
        X = rng.standard_normal((n, m)) * (1.0 + np.arange(m)) / m
        Xd = to_dev(X, ld=ld)
        G = _noalloc(H, Xd, n, m, ld)
        ref = oracle.gram(X)
        assert np.all(np.isfinite(G)), (n, m)
        assert np.all(np.abs(G - ref) <= _gram_tol(ref, n)), (n, m)
        # and the same matrix as the entry point that allocates its workspace
        G2 = H.hapod_gram(Xd, H.HAPOD_FP64).cpu().numpy()
        assert np.all(np.abs(G - G2) <= _gram_tol(ref, n)), (n, m)


def test_noalloc_gram_no_rows_gives_zero(cuda_ok):
    from paper_1607_05210_gb300 import hapod as H

    X = torch.zeros((5, 1), dtype=torch.float64, device="cuda")
    G = _noalloc(H, X, 0, 5, 1)
    assert np.array_equal(G, np.zeros((5, 5)))


def test_noalloc_gram_rejects_too_wide(cuda_ok):
    from paper_1607_05210_gb300 import hapod as H

    X = to_dev(np.ones((1, 2900)))
    G = torch.empty((2900, 2900), dtype=torch.float64, device="cuda")
    st = H._lib.hapod_gram_noalloc(1, 2900, ctypes.c_void_p(X.data_ptr()), 1, ctypes.c_void_p(G.data_ptr()), None)
    assert st == H.HAPOD_ERR_INVALID
    assert "2816" in H.hapod_last_error()
