"""The batched uneven workload: leaves of the prescribed-spectrum generator with
column counts m_l ~ U{16..512} and decay rates delta_l ~ U[1/40, 1/10] decades per
index over a shared basis, balanced quaternary tree, eps = 1e-5 rel, omega = 0.5; every
level (every batch of ready nodes, uneven m) runs as one grouped launch per step.

Against the CPU oracle on the same values (tests/tree_check.py), at sizes the oracle
finishes in about a minute:
  * the first 16 leaves of the workload's own draw (m in [16, 512], shared rank 200)
    at n = 1024 rows, as the level-3 subtree they form in the workload's tree;
  * 64 leaves with m ~ U{16..96} over a shared rank-60 basis at n = 2048 rows on a
    quaternary tree of depth 3 (L_T = 4): three levels of uneven grouped batches.
Full size in the launch configuration bench.py times (n = 2^18, 1000 leaves, 278 GB
generated on the device in waves of 64 leaves), where the oracle cannot follow: the
properties of tree_check.full_size_waves.
"""
import numpy as np
import pytest

from paper_1607_05210_gb300 import synth
from tests import tree_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def _data(seed, n, m, delta, rank, parent):
    leaves = synth.leaves_of(parent)
    Q = synth.shared_basis(seed, n, rank)
    cols = [0] * len(parent)
    data = {}
    for i, a in enumerate(leaves):
        cols[a] = int(m[i])
        data[a] = synth.uneven_leaf(Q, seed, i, int(m[i]), float(delta[i]), dtype=np.float32).astype(np.float64)
    X = np.asfortranarray(np.concatenate([data[a] for a in leaves], axis=1))
    return cols, data, X


@pytest.fixture(scope="module", params=["draw16_n1024", "narrow64_n2048"])
def reduced(request):
    import bench

    seed = bench.C4["seed"]
    if request.param == "draw16_n1024":
        n, parent = 1024, synth.balanced_tree(4, 2)
        m = synth.uneven_leaf_cols(seed, 16, 16, 512)
        delta = synth.uneven_decays(seed, 16)
        rank = 200
    else:
        n, parent = 2048, synth.balanced_tree(4, 3)
        m = synth.uneven_leaf_cols(seed + 7, 64, 16, 96)
        delta = synth.uneven_decays(seed + 7, 64)
        rank = 60
    cols, data, X = _data(seed, n, m, delta, rank, parent)
    eps = 1e-5 * float(np.linalg.norm(X))
    return request.param, n, parent, cols, data, X, eps, tree_check.oracle_tree(parent, cols, data, eps, 0.5)


@pytest.mark.parametrize("form", ["fx3", "fp64_ozaki"])
def test_uneven_leaves_against_oracle(H, reduced, form):
    name, n, parent, cols, data, X, eps, ora = reduced
    prec = H.HAPOD_MIXED_FX3 if form == "fx3" else H.HAPOD_FP64_OZAKI
    gpu = tree_check.hapod_gpu(H, prec, parent, cols, data, n, eps, 0.5)
    assert gpu[3] in (H.HAPOD_OK, H.HAPOD_WARN_BELOW_FLOOR)
    tree_check.check(H, prec, parent, cols, data, X, eps, 0.5, gpu, ora, 1e-5 if form == "fx3" else None,
                     label=f"{name} {form}")


def test_uneven_leaves_full_size(H):
    import bench

    tree_check.full_size_waves(H, bench, bench.C4)
