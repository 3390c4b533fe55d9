"""The Gram schedule autotuner (hapod_autotune): it times the candidate split
factors on the caller's node, keeps the fastest for the node's (form, m, n) bucket,
and every later Gram in that bucket uses it.  The Gram stays what the form's
arithmetic makes it whatever the split count: checked against the oracle under each
factor with the form's own bound (the row splits only regroup exact per-split sums
added in FP64)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    yield hapod
    hapod.hapod_autotune_clear()


@pytest.mark.parametrize("form,n,m", [("fx3", 1 << 17, 128), ("fx3", 1 << 16, 300), ("fp64", 1 << 15, 100),
                                      ("bf16x3", 1 << 16, 128)])
def test_autotune_keeps_the_gram(H, form, n, m):
    prec = {"fx3": H.HAPOD_MIXED_FX3, "fp64": H.HAPOD_FP64, "bf16x3": H.HAPOD_MIXED_BF16X3}[form]
    X = synth.advection_pulses(n, m, 5).astype(np.float32).astype(np.float64)
    Xd = to_dev(X, dtype=H.DTYPE[prec])
    pct, ms = H.hapod_autotune(Xd, prec)
    print(f"{form} n={n} m={m}: factor {pct} %, ms {[round(v, 3) for v in ms]}")
    assert pct in (50, 100, 200, 400)
    assert all(v > 0 for v in ms)
    assert ms[[50, 100, 200, 400].index(pct)] <= min(ms) / 0.98 + 1e-9
    ref = oracle.gram(X)
    d = np.sqrt(np.diag(ref))
    tol = {"fx3": 1e-9, "fp64": 1e-13 * math.sqrt(n), "bf16x3": 1e-5}[form]
    G = H.hapod_gram(Xd, prec).cpu().numpy()
    assert np.max(np.abs(G - ref) / np.outer(d, d)) <= tol
    H.hapod_autotune_clear()
    G2 = H.hapod_gram(Xd, prec).cpu().numpy()
    assert np.max(np.abs(G2 - ref) / np.outer(d, d)) <= tol


def test_autotune_rejects_other_forms(H):
    X = to_dev(np.ones((1000, 4)))
    with pytest.raises(H.HapodError) as e:
        H.hapod_autotune(X, H.HAPOD_FP64_OZAKI)
    assert e.value.status == H.HAPOD_ERR_INVALID
