"""The streamed incremental workload (Sec. 3.2 skinny tree, Sec. 3.4 reduced memory):
snapshots in chunks of 64 columns pushed as they are generated, on a left-deep chain
of four binary subtrees of depth 4 (L_T = 8), eps = 1e-4 rel, omega = 0.5, on the
mixed fixed-point form and on the digit-slice FP64 form.

Reduced size against the CPU oracle on the same values (tests/tree_check.py): the
same tree and chunk width at n = 2048 rows, pushed in the streaming order (subtree 1
first) with 8 chunks pending at most.  Full size in the launch configuration
bench.py times (n = 2^23, 64 chunks generated on the device, 8 resident), where the
oracle cannot follow: the properties of tree_check.full_size_waves.
"""
import numpy as np
import pytest

from paper_1607_05210_gb300 import synth
from tests import tree_check
from tests.helpers import leaf_split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


@pytest.fixture(scope="module")
def reduced():
    import bench

    wl = dict(bench.C5, n=2048)
    parent, leaves, cols = bench.c3_tree(wl)
    S = sum(cols)
    X = synth.pulse_snapshots(wl["n"], 0, S, synth.pulse_workload(wl["seed"]), np.float32).astype(np.float64)
    data, off = {}, 0
    for a in leaves:  # chunk i -> leaf i of the streaming order
        data[a] = np.asfortranarray(X[:, off:off + cols[a]])
        off += cols[a]
    eps = wl["eps_rel"] * float(np.linalg.norm(X))
    return wl, parent, cols, data, X, eps, tree_check.oracle_tree(parent, cols, data, eps, wl["omega"])


@pytest.mark.parametrize("form", ["fx3", "fp64_ozaki"])
def test_streamed_chain_against_oracle(H, reduced, form):
    wl, parent, cols, data, X, eps, ora = reduced
    prec = H.HAPOD_MIXED_FX3 if form == "fx3" else H.HAPOD_FP64_OZAKI
    gpu = tree_check.hapod_gpu(H, prec, parent, cols, data, wl["n"], eps, wl["omega"], max_pending=wl["wave"])
    assert gpu[3] == H.HAPOD_OK
    tree_check.check(H, prec, parent, cols, data, X, eps, wl["omega"], gpu, ora, 1e-5 if form == "fx3" else None,
                     label=f"chain {form}")


def test_streamed_chain_full_size(H):
    import bench

    tree_check.full_size_waves(H, bench, bench.C5)
