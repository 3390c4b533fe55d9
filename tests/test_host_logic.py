"""Host-side helpers of the sweeps (no GPU): the tree-shape builder of Sec. 4.2 and
the direct-POD rank used to count additional HAPOD modes (Sec. 4.3)."""
import json
import math

import numpy as np
import pytest

import bench
import oracle
from paper_1607_05210_gb300 import synth


def _depths(parent):
    d = []
    for a in range(len(parent)):
        k, b = 0, a
        while parent[b] >= 0:
            b = parent[b]
            k += 1
        d.append(k)
    return d


@pytest.mark.parametrize("blocks,depth", [(10, 2), (40, 2), (100, 2), (100, 3), (400, 4), (1000, 5), (1, 3), (64, 6)])
def test_nary_tree_shape(blocks, depth):
    """s blocks on the first leaf slots of a balanced n-ary tree of the given edge
    depth, n the smallest arity with n^depth >= s; one root, every leaf at the full
    depth, no inner node without a leaf below it."""
    parent = synth.nary_tree(blocks, depth)
    leaves = synth.leaves_of(parent)
    assert len(leaves) == blocks
    assert parent.count(-1) == 1
    arity = next(a for a in range(1, blocks + 2) if a ** depth >= blocks)
    kids = [0] * len(parent)
    for p in parent:
        if p >= 0:
            kids[p] += 1
    assert max(kids) == (arity if blocks > 1 else 1)
    d = _depths(parent)
    assert all(d[a] == depth for a in leaves)
    assert all(kids[a] > 0 for a in range(len(parent)) if a not in set(leaves))


def test_nary_tree_matches_the_benchmark_tree():
    """64 blocks at edge depth 6 is the benchmark's balanced binary tree."""
    assert synth.nary_tree(64, 6) == synth.balanced_tree(2, 6)


@pytest.mark.parametrize("seed", range(6))
def test_direct_pod_rank_matches_oracle_truncation(seed):
    """The bench's rank from a spectrum equals the oracle's POD rank (Def. truncated
    POD, inclusive threshold) on a matrix with that spectrum."""
    rng = np.random.default_rng(seed)
    m = 12
    sigma = np.sort(rng.uniform(0.0, 1.0, m) ** 3)[::-1]
    X = np.zeros((20, m))
    X[:m, :m] = np.diag(sigma)
    for eps in (0.0, 1e-3, float(sigma[m // 2]), 0.3, 10.0):
        k_ref = oracle.pod(X, eps).N if eps > 0 else m
        assert bench.direct_pod_rank(sigma, eps) == k_ref


def test_direct_pod_rank_inclusive_threshold():
    # tail after keeping 1 is exactly eps^2: keep 1 (the comparison is <=)
    assert bench.direct_pod_rank([2.0, 1.0], 1.0) == 1
    assert bench.direct_pod_rank([2.0, 1.0], 0.999) == 2
    assert bench.direct_pod_rank([2.0, 1.0], math.sqrt(5.0)) == 0


def test_roofline_fields_for_the_digit_slice_gram():
    """bench.py's roofline object: the digit Gram step on the method's algorithmic bytes
    (8 n m per node) against the measured HBM peak, the digit-pair tensor rate beside
    it, and traffic either a recorded capture of the unchanged kernel or null."""
    from paper_1607_05210_gb300 import hapod as H

    res = {"steps": {"gram": {"ms": 100.0, "launches": 64, "bytes": 1e9, "flops": 2e12},
                     "modes": {"ms": 50.0, "launches": 7, "bytes": 1e9, "flops": 1e11}}}
    dom, roof = bench.roofline(res, H.HAPOD_FP64_OZAKI, H, 6786.2)
    assert dom == "gram" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(1e9 / 0.1 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6786.2)
    assert roof["digit_tflops"] == pytest.approx(28 * 2e12 / 0.1 / 1e12)
    assert roof["traffic"] is None or (isinstance(roof["traffic"], float) and roof["traffic"] > 0)


def test_kernel_traffic_is_null_once_the_source_changed(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    import hashlib

    rec = {"k": {"source": str(src), "sha256": hashlib.sha256(b"kernel v1").hexdigest(),
                 "bytes_per_launch": 5.0e9, "note": "capture"}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.kernel_traffic("k") == (5.0e9, "capture")
    src.write_text("kernel v2")
    assert bench.kernel_traffic("k")[0] is None
    assert bench.kernel_traffic("missing")[0] is None


def test_mixed_gram_roofline_is_hbm_bound():
    from paper_1607_05210_gb300 import hapod as H

    res = {"steps": {"gram": {"ms": 100.0, "launches": 64, "bytes": 1e9, "flops": 2e12},
                     "modes": {"ms": 50.0, "launches": 7, "bytes": 1e9, "flops": 1e11}}}
    for prec in (H.HAPOD_MIXED_TF32X3, H.HAPOD_MIXED_FX3, H.HAPOD_MIXED_BF16X3):
        dom, roof = bench.roofline(res, prec, H, 6786.2, "gram")
        assert roof["bound"] == "hbm" and roof["achieved"] == pytest.approx(1e9 / 0.1 / 1e9)
        assert roof["frac"] == pytest.approx(10.0 / 6786.2)
    assert bench.roofline(res, H.HAPOD_MIXED_FX3, H, 6786.2, "gram")[1]["kernel"] == "gram_fx3_kernel"


def test_headline_tree_and_workload():
    """The precision workload's tree: balanced quaternary of edge depth 4 (L_T = 5),
    256 leaves x 128 columns, waves of 16 leaves = whole level-3 subtrees."""
    parent, leaves, cols = bench.c3_tree()
    assert len(leaves) == 256 and sum(cols) == 32768 and len(parent) == 341
    levels = oracle.tree_levels(parent)
    assert max(levels) == 5
    W = bench.C3["wave"]
    for w0 in range(0, 256, W):
        anc = set()
        for a in leaves[w0:w0 + W]:
            anc.add(parent[parent[a]])
        assert len(anc) == 1  # one level-3 node per wave


def test_rank_within_accepts_only_ranks_of_nearby_tolerances():
    from tests.helpers import rank_within

    tails = np.array([10.0, 4.0, 1.0, 0.5, 0.0])  # sum_{i >= j} sigma_i^2
    eps = 1.0
    assert rank_within(2, tails, eps, 0.0)           # the exact rank (inclusive threshold)
    assert not rank_within(1, tails, eps, 0.0)
    assert not rank_within(3, tails, eps, 0.0)
    assert rank_within(3, tails, eps, 0.01)          # tails[2] = eps^2 within delta
    assert not rank_within(4, tails, eps, 0.01)
    assert rank_within(1, tails, math.sqrt(4.0), 0.0) and not rank_within(0, tails, 2.0, 0.0)
