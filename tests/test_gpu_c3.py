"""The precision workload (travelling pulses, quaternary tree, eps = 1e-4 rel, omega =
0.5) on the mixed fixed-point form and on the digit-slice FP64 form.

Reduced sizes, against the CPU oracle run on the same values (tests/tree_check.py):
  * the workload's tree shape: balanced quaternary tree of edge depth 4 (L_T = 5,
    256 leaves, 341 nodes) with 16 snapshots per leaf at n = 4096 rows;
  * the workload's leaf width: 128 snapshots per leaf on a quaternary tree of edge
    depth 2 (16 leaves) at n = 2^14 rows.
Full size, in the launch configuration bench.py times (n = 2^22, 256 leaves x 128
snapshots generated on the device in waves of 16 leaves, max_pending_leaves = 16),
where the oracle cannot follow: properties that hold at any size -- the projection
error of each form's root modes within Thm. hapod_bound's sum of eps(a)^2 (computed
leaf by leaf from regenerated snapshots in FP64 as ||X||^2 - ||Q^T X||^2, Q an
orthonormal basis of the modes), and the two forms' ranks and singular values
agreeing within the fixed-point form's measured Gram error on a full-size leaf.
"""
import math

import numpy as np
import pytest
import torch

from paper_1607_05210_gb300 import synth
from tests import tree_check
from tests.helpers import leaf_split

pytestmark = pytest.mark.gpu

SEED = 1607052103


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def _workload(n, cols_per_leaf, depth):
    parent = synth.balanced_tree(4, depth)
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = cols_per_leaf
    S = sum(cols)
    X = synth.pulse_snapshots(n, 0, S, synth.pulse_workload(SEED), np.float32).astype(np.float64)
    _, data = leaf_split(X, parent, cols)
    eps = 1e-4 * float(np.linalg.norm(X))
    return parent, cols, data, X, eps


@pytest.fixture(scope="module", params=[(4096, 16, 4), (1 << 14, 128, 2)], ids=["shape_LT5", "width128_LT3"])
def reduced(request):
    n, c, depth = request.param
    parent, cols, data, X, eps = _workload(n, c, depth)
    return parent, cols, data, X, eps, tree_check.oracle_tree(parent, cols, data, eps, 0.5), n


@pytest.mark.parametrize("form", ["fx3", "fp64_ozaki"])
def test_precision_workload_against_oracle(H, reduced, form):
    parent, cols, data, X, eps, ora, n = reduced
    prec = H.HAPOD_MIXED_FX3 if form == "fx3" else H.HAPOD_FP64_OZAKI
    gpu = tree_check.hapod_gpu(H, prec, parent, cols, data, n, eps, 0.5, max_pending=16)
    assert gpu[3] == H.HAPOD_OK
    tree_check.check(H, prec, parent, cols, data, X, eps, 0.5, gpu, ora, 1e-5 if form == "fx3" else None,
                     label=f"{form} n={n}")


# ------------------------------------------------------------------ full size
def test_precision_workload_full_size(H):
    import bench

    tree_check.full_size_waves(H, bench, bench.C3)
