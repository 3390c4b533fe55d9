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
def _full_size_run(H, bench, precision, fro2, stream):
    """bench.run_waves' schedule, returning the root modes too."""
    wl = bench.C3
    parent, leaves, cols = bench.c3_tree(wl)
    device = torch.device("cuda", 0)
    gen = bench.Generator(H, wl, H.DTYPE[precision], device, wl["wave"])
    eps = wl["eps_rel"] * math.sqrt(fro2)
    ctx = H.hapod_create(parent, cols, eps, wl["omega"], wl["n"], precision, stream=stream,
                         max_pending_leaves=wl["wave"])
    with torch.cuda.stream(stream):
        for w0 in range(0, len(leaves), wl["wave"]):
            for i in range(w0, w0 + wl["wave"]):
                gen.gen(i, i - w0, stream)
            for i in range(w0, w0 + wl["wave"]):
                H.hapod_push(ctx, leaves[i], gen.bufs[i - w0].t())
        s, U, st = H.hapod_result(ctx, device=device)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    del gen
    torch.cuda.synchronize()
    return s.numpy(), U, stats, st


def _projection_error(H, bench, U):
    """sum over all snapshots of ||x - Q Q^T x||^2 = ||X||^2 - ||Q^T X||^2 in FP64, Q
    from a QR of the modes (FP64 accumulation; the cancellation costs about 8 of 16
    digits at a relative error of 1e-8)."""
    wl = bench.C3
    Q, _ = torch.linalg.qr(U.double())
    gen = bench.Generator(H, wl, torch.float32, U.device, 1)
    cur = torch.cuda.current_stream()
    tot = 0.0
    for i in range(wl["leaves"]):
        X = gen.gen(i, 0, cur).double()  # cols x n
        C = X @ Q                        # cols x k = (Q^T X)^T
        tot += float(torch.sum(X * X) - torch.sum(C * C))
    torch.cuda.synchronize()
    return tot


def test_precision_workload_full_size(H):
    import bench
    import oracle

    stream = torch.cuda.Stream()
    wl = bench.C3
    fro2 = bench.c3_fro2(H, wl, torch.device("cuda", 0), stream)
    parent, leaves, cols = bench.c3_tree(wl)
    eps = wl["eps_rel"] * math.sqrt(fro2)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(sum(cols)), wl["omega"])
    bound = sum(e * e for e in eps_nodes)
    res = {}
    for form, prec in (("fx3", H.HAPOD_MIXED_FX3), ("fp64_ozaki", H.HAPOD_FP64_OZAKI)):
        s, U, stats, st = _full_size_run(H, bench, prec, fro2, stream)
        assert st == H.HAPOD_OK, form
        assert all(stats[a]["tail_sq"] <= eps_nodes[a] ** 2 * (1 + 1e-12) for a in range(len(parent))), form
        perr = _projection_error(H, bench, U)
        print(f"{form}: k_root={len(s)} projection error {perr / bound:.4f} of the bound, "
              f"{perr / fro2:.3e} of ||X||^2")
        assert perr <= bound * 1.01, form
        res[form] = (s, stats)
        del U
        torch.cuda.empty_cache()
    # the fixed-point form's Gram error on a full-size leaf, against the digit-slice
    # FP64 Gram of the same values (exact to FP64 rounding)
    gen = bench.Generator(H, wl, torch.float32, torch.device("cuda", 0), 1)
    X = gen.gen(0, 0, torch.cuda.current_stream()).t()
    G1 = H.hapod_gram(X, H.HAPOD_MIXED_FX3)
    G2 = H.hapod_gram(X.double(), H.HAPOD_FP64_OZAKI)
    e_leaf = float(torch.linalg.matrix_norm(G1 - G2, ord=2))
    tr_leaf = float(torch.trace(G2))
    del gen, X
    u_eff = e_leaf / tr_leaf  # per unit of trace; every node's Gram error scales with its trace
    (s1, st1), (s2, st2) = res["fx3"], res["fp64_ozaki"]
    differ = [a for a in range(len(parent)) if st1[a]["k"] != st2[a]["k"]]
    print(f"u_eff={u_eff:.2e}; nodes with other rank: {len(differ)} of {len(parent)}; "
          f"k_root {len(s1)} / {len(s2)}")
    assert all(abs(st1[a]["k"] - st2[a]["k"]) <= 1 for a in differ)
    assert abs(len(s1) - len(s2)) <= 1
    k = min(len(s1), len(s2))
    slack = math.sqrt(sum(eps_nodes[a] ** 2 for a in differ if parent[a] >= 0))
    dsig = np.abs(s1[:k] - s2[:k])
    assert np.all(dsig <= 10 * u_eff * len(parent) * fro2 / s2[:k] + 1e-6 * s2[0] + slack), dsig.max()
