"""Low-rank approximation of the snapshot map (Sec. 3.3, Remark "Low-rank
approximation of the snapshot mapping", Eq. low_rank_approx): with the right factor
Lambda~ of hapod_result_right,

    || S - U diag(sigma) Lambda~^T ||_F^2 <= sum over all nodes a of eps(a)^2,

Lambda~ with orthonormal columns (a product of block-diagonal matrices with
orthonormal columns, Def. "Additional notation").  Checked on star, binary,
incremental-chain and quaternary trees for the FP64, digit-slice and fixed-point
forms, with a pass-through leaf (eps = 0: identity) and a leaf that keeps no mode
(its rows are zero); on a single node the approximation equals the oracle's
truncated SVD U_N diag(sigma) V_N^T (no tie at the cut).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import leaf_split, to_dev, to_host

pytestmark = pytest.mark.gpu

TREES = {"star": synth.star_tree(5), "binary": synth.balanced_tree(2, 3), "chain": synth.chain_of_subtrees(3, 1),
         "quaternary": synth.balanced_tree(4, 2)}


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def _run(H, precision, parent, cols, X, eps, override=None):
    leaves, data = leaf_split(X, parent, cols)
    dtype = H.DTYPE[precision]
    ctx = H.hapod_create(parent, cols, eps, 0.5, X.shape[0], precision, eps_override=override,
                         flags=H.HAPOD_FLAG_RIGHT_VECTORS)
    bufs = {a: to_dev(data[a], dtype=dtype) for a in leaves}
    for a in leaves:
        H.hapod_push(ctx, a, bufs[a])
    s, U, st = H.hapod_result(ctx)
    W = H.hapod_result_right(ctx, len(s))
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    return s.numpy(), to_host(U), to_host(W), stats, st


@pytest.mark.parametrize("special", ["plain", "passthrough_and_dropped"])
@pytest.mark.parametrize("form", ["fp64", "fp64_ozaki", "fx3"])
@pytest.mark.parametrize("tree", sorted(TREES))
def test_low_rank_approximation_bound(H, form, tree, special):
    parent = TREES[tree]
    leaves = synth.leaves_of(parent)
    rng = np.random.default_rng(len(parent))
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(20, 70))
    S = sum(cols)
    if form == "fx3":
        X = synth.advection_pulses(1 << 13, S, S).astype(np.float32).astype(np.float64)
        rel = 1e-4
    else:
        X = synth.prescribed_spectrum(3000, S, 10.0 ** (-np.arange(min(S, 120)) / 12.0), seed=S, noise=1e-12)
        rel = 1e-6
    X = np.asfortranarray(X)
    prec = {"fp64": H.HAPOD_FP64, "fp64_ozaki": H.HAPOD_FP64_OZAKI, "fx3": H.HAPOD_MIXED_FX3}[form]
    eps = rel * float(np.linalg.norm(X))
    override = None
    if special != "plain":
        # leaf 0 passes its snapshots through (eps = 0), the last leaf keeps no mode
        override = [float("nan")] * len(parent)
        override[leaves[0]] = 0.0
        Xl = X[:, sum(cols[a] for a in leaves[:-1]):]
        override[leaves[-1]] = 2.0 * float(np.linalg.norm(Xl))
    s, U, W, stats, st = _run(H, prec, parent, cols, X, eps, override)
    k = len(s)
    assert W.shape == (S, k)
    if override is not None:
        assert stats[leaves[0]]["k"] == cols[leaves[0]] and stats[leaves[-1]]["k"] == 0
        assert np.all(W[S - cols[leaves[-1]]:] == 0.0)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), 0.5)
    for a, v in enumerate(override or []):
        if not math.isnan(v):
            eps_nodes[a] = v
    bound = sum(e * e for e in eps_nodes)
    R = X - (U * s) @ W.T
    err = float(np.sum(R * R))
    ortho = float(np.max(np.abs(W.T @ W - np.eye(k))))
    print(f"{tree} {form} {special}: k={k} error {err / bound:.3f} of the bound, |W^T W - I| = {ortho:.1e}")
    assert err <= bound * 1.01
    assert ortho <= 1e-10


@pytest.mark.parametrize("form", ["fp64", "fp64_ozaki"])
def test_single_node_is_the_truncated_svd(H, form):
    n, m = 2000, 60
    X = synth.prescribed_spectrum(n, m, 10.0 ** (-np.arange(m) / 10.0), seed=3)
    sig = np.linalg.svd(X, compute_uv=False)
    eps = float(np.sqrt(np.sum(sig[25:] ** 2)) * 1.001)  # cut inside the gap after 25 modes
    prec = H.HAPOD_FP64 if form == "fp64" else H.HAPOD_FP64_OZAKI
    s, U, W, stats, st = _run(H, prec, [-1], [m], X, eps)
    assert len(s) == 25
    s_o, US_o, V_o, _ = oracle.svd(X)  # US_o = U_o diag(sigma), V_o m x r
    ref = US_o[:, :25] @ V_o[:, :25].T
    diff = float(np.linalg.norm((U * s) @ W.T - ref))
    print(f"single node {form}: |U S W^T - U_o S_o V_o^T| = {diff:.2e} of |X| {np.linalg.norm(X):.2e}")
    assert diff <= 1e-8 * float(np.linalg.norm(X))


def test_requires_the_flag(H):
    X = to_dev(np.ones((100, 3)))
    ctx = H.hapod_create([-1], [3], 1e-3, 0.5, 100, H.HAPOD_FP64)
    H.hapod_push(ctx, 0, X)
    s, U, st = H.hapod_result(ctx)
    with pytest.raises(H.HapodError) as e:
        H.hapod_result_right(ctx, len(s))
    assert e.value.status == H.HAPOD_ERR_STATE
    H.hapod_destroy(ctx)
