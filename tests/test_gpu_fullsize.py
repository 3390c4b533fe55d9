"""The benchmark workload at full size, in the launch configuration bench.py times.

n = 2^20 rows, 64 leaves x 256 advection-diffusion snapshots (137 GB FP64 on the
device), balanced binary tree L_T = 7 (and the two-level star), eps = 1e-5 ||X||_F, omega = 0.5, the
digit-slice FP64 form, every leaf pushed and then processed in one batch, as in
the bench's timed step.

The oracle cannot take the POD of 2^20-row matrices in seconds, but these
snapshots have a closed form: X = B C with B = [sin(k x_i), cos(k x_i)], k = 1..32,
whose columns are orthogonal with squared norm n/2 on the uniform grid.  Every
node input is then S~_a = B K_a (the outputs of the children stay in span(B)), and
S~_a has the singular values and the right singular vectors of sqrt(n/2) K_a
(64 x m_a).  The oracle's HAPOD recursion (Def. HAPOD) run on the leaves
sqrt(n/2) C_a therefore takes the same ranks and singular values as the full-size
HAPOD, node by node, and its root modes, mapped back through B / sqrt(n/2), are
the full-size modes.  Checked: every node's rank (up to a genuine tie at eps(a)^2),
the root's singular values (1e-6 relative above 1e-5 sigma_max) and the largest
principal angle between the GPU's and the oracle's root modes.  The same check
runs for other omega (Sec. 4.3) and for the tree shapes of Sec. 4.2 (10^4 columns
in blocks on balanced n-ary trees, at n = 2^14 rows).
"""
import math

import numpy as np
import pytest
import torch

import bench
import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import max_angle_sin, rank_agrees, sigma_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    bufs, fro2 = bench.make_inputs(torch.float64, torch.device("cuda", 0))
    yield bufs, fro2
    del bufs
    torch.cuda.empty_cache()


def _run(H, parent, leaves, cols, bufs, n, eps, omega):
    device = bufs[0].device
    ctx = H.hapod_create(parent, cols, eps, omega, n, H.HAPOD_FP64_OZAKI, stream=torch.cuda.Stream(device))
    for i, a in enumerate(leaves):
        H.hapod_push(ctx, a, bufs[i].t())
    s, U, st = H.hapod_result(ctx, device=device)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    assert st == H.HAPOD_OK
    return s.numpy(), U, stats


def _closed_form_check(parent, leaves, cols, C, n, eps, omega, s, stats):
    """The oracle's HAPOD on sqrt(n/2) C_a; ranks of every node and root sigma."""
    S = sum(cols)
    scale = math.sqrt(n / 2.0)
    data, off = {}, 0
    for a in leaves:
        data[a] = scale * C[:, off:off + cols[a]]
        off += cols[a]
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), omega)
    ref = oracle.hapod(parent, data, eps_nodes, keep_all=True)
    children = [[b for b in range(len(parent)) if parent[b] == a] for a in range(len(parent))]
    for a in range(len(parent)):
        X_a = data[a] if not children[a] else np.concatenate([ref[b].Y for b in children[a]], axis=1)
        tails = oracle.tail_sums(oracle.svd(X_a, want_vectors=False)[0])
        assert rank_agrees(stats[a]["k"], ref[a].N, tails, eps_nodes[a]), (a, stats[a]["k"], ref[a].N)
    root = parent.index(-1)
    ok, err = sigma_close(s, ref[root].sigma, 1e-6, 1e-5)
    assert ok, err
    return ref, children, root


@pytest.mark.parametrize("kind", ["binary", "star"])
def test_bench_workload_against_closed_form_oracle(workload, kind):
    """The FP64 workload on both of its trees: the balanced binary tree (L_T = 7) and
    the two-level star (L_T = 2), whose root sees every leaf's modes at once."""
    from paper_1607_05210_gb300 import hapod as H

    bufs, fro2 = workload
    device = bufs[0].device
    parent, leaves, cols = bench.tree(kind)
    n, S = bench.N_ROWS, bench.LEAVES * bench.COLS
    eps = bench.EPS_REL * math.sqrt(fro2)
    s, U, stats = _run(H, parent, leaves, cols, bufs, n, eps, bench.OMEGA)
    C = synth.advection_diffusion_coeffs(S, bench.SEED)
    ref, children, root = _closed_form_check(parent, leaves, cols, C, n, eps, bench.OMEGA, s, stats)

    # root modes: U_ref = (B / sqrt(n/2)) (Y_c / sigma), compared by principal angles
    scale = math.sqrt(n / 2.0)
    k = min(U.shape[1], ref[root].N)
    B = torch.from_numpy(synth.fourier_basis(n)).to(device)
    W = torch.from_numpy(np.ascontiguousarray(ref[root].Y[:, :k] / ref[root].sigma[:k])).to(device) / scale
    U_ref = np.linalg.qr((B @ W).cpu().numpy())[0]
    U_gpu = np.linalg.qr(U[:, :k].double().cpu().numpy())[0]
    del B
    # an FP64 Gram-based mode is accurate to ~u (sigma_1 / sigma_j)^2; against the
    # gap to the first discarded singular value of the root's input
    X_root = np.concatenate([ref[b].Y for b in children[root]], axis=1)
    sig_root = oracle.svd(X_root, want_vectors=False)[0]
    gap = sig_root[k - 1] ** 2 - (sig_root[k] ** 2 if sig_root.size > k else 0.0)
    tol = 1e-6 * sig_root[0] ** 2 / gap
    assert max_angle_sin(U_gpu, U_ref) <= tol


@pytest.mark.parametrize("omega", [0.1, 0.95])
def test_bench_workload_other_omega(workload, omega):
    """Sec. 4.3's trade-off parameter: smaller omega gives more final modes."""
    from paper_1607_05210_gb300 import hapod as H

    bufs, fro2 = workload
    parent, leaves, cols = bench.tree()
    n, S = bench.N_ROWS, bench.LEAVES * bench.COLS
    eps = bench.EPS_REL * math.sqrt(fro2)
    s, U, stats = _run(H, parent, leaves, cols, bufs, n, eps, omega)
    C = synth.advection_diffusion_coeffs(S, bench.SEED)
    _closed_form_check(parent, leaves, cols, C, n, eps, omega, s, stats)


@pytest.mark.parametrize("blocks,edge_depth", [(40, 2), (100, 3), (400, 4), (1000, 5)])
def test_tree_shapes_against_closed_form_oracle(blocks, edge_depth):
    """Sec. 4.2's tree shapes: 10^4 columns in `blocks` equal blocks on the balanced
    n-ary tree of the given edge depth, n = 2^14 rows."""
    from paper_1607_05210_gb300 import hapod as H

    n, total = 1 << 14, 10_000
    c = total // blocks
    device = torch.device("cuda", 0)
    Xt = synth.advection_diffusion_device(n, total, bench.SEED, torch.float64, device)
    fro2 = float(torch.sum(Xt * Xt))
    parent = synth.nary_tree(blocks, edge_depth)
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = c
    bufs = [Xt[i * c:(i + 1) * c] for i in range(blocks)]
    eps = bench.EPS_REL * math.sqrt(fro2)
    s, U, stats = _run(H, parent, leaves, cols, bufs, n, eps, bench.OMEGA)
    C = synth.advection_diffusion_coeffs(total, bench.SEED)
    _closed_form_check(parent, leaves, cols, C, n, eps, bench.OMEGA, s, stats)
