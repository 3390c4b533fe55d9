"""Mixed form (FP32 snapshots; tcgen05 TF32x3 Gram, FP32 CUDA-core modes,
FP32 Jacobi with FP64 Rayleigh quotients, FP64 truncation) versus the CPU FP64
oracle run on the same FP32 values.

Tolerances, derived from the arithmetic:
  * Gram: hi = x truncated to TF32 (10 mantissa bits), lo = x - hi, read by the
    tensor core truncated to TF32 again, so |x - hi - lo_tf32| <= 2^-20 |x|; the
    dropped lo*lo term is <= 2^-20 |x_i x_j|; the FP32 tensor accumulation of one
    64-row segment (24 truncating steps) adds <= 24 * 2^-23 of the segment's
    magnitude; with Cauchy-Schwarz, |G - G_ref| <= 1e-5 sqrt(G_ii G_jj).
  * singular values: |d sigma_j| <= 10 u_eff ||X||_F^2 / sigma_j with u_eff = 2e-5
    (eigenvalue perturbation by the Gram error), checked above the floor.
  * ranks: equal except near-ties; projection error within Thm. hapod_bound with a
    stated 1 % slack.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import leaf_split, projection_error, rank_agrees, to_dev, to_host

pytestmark = pytest.mark.gpu
U_EFF = 1e-5


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def _f32(X):
    return np.asfortranarray(np.asarray(X, dtype=np.float32).astype(np.float64))


@pytest.mark.parametrize("n,m,ld,kind", [(1000, 1, 1000, "gauss"), (10000, 100, 10000, "gauss"),
                                         (3000, 130, 3001, "gauss"), (50000, 256, 50000, "smooth"),
                                         (70, 200, 72, "gauss"), (200000, 300, 200000, "smooth"),
                                         (64, 128, 64, "gauss"), (131072, 128, 131072, "smooth")])
def test_gram_mixed(H, n, m, ld, kind):
    rng = np.random.default_rng(n + m)
    if kind == "gauss":
        X = rng.standard_normal((n, m)) * (1.0 + np.arange(m)) / m
    else:
        X = synth.advection_diffusion(n, m, seed=m)
    X = _f32(X)
    G = H.hapod_gram(to_dev(X, dtype=torch.float32, ld=ld), H.HAPOD_MIXED_TF32X3).cpu().numpy()
    ref = oracle.gram(X)
    d = np.sqrt(np.diag(ref))
    scale = np.outer(d, d)
    rel = np.abs(G - ref) / np.maximum(scale, 1e-300)
    print(f"gram mixed n={n} m={m} {kind}: max {rel.max():.3e} rms {np.sqrt(np.mean(rel ** 2)):.3e}")
    assert np.all(np.abs(G - ref) <= U_EFF * scale)
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("n,m,N", [(1000, 100, 37), (4097, 130, 20), (300, 1, 1), (12345, 64, 64), (9999, 256, 70)])
def test_modes_mixed(H, n, m, N):
    rng = np.random.default_rng(n)
    X = _f32(rng.standard_normal((n, m)))
    V = np.asfortranarray(rng.standard_normal((m, N)))
    scale = rng.uniform(0.5, 2.0, N)
    Y = to_host(H.hapod_modes(to_dev(X, dtype=torch.float32), to_dev(V), N, torch.from_numpy(scale).cuda(),
                              H.HAPOD_MIXED_TF32X3))
    Vf = V.astype(np.float32).astype(np.float64)  # V is rounded to FP32 once
    ref = (X @ Vf) * scale
    # FP32 FMA chain of length m plus the FP32 rounding of the output
    bound = (m + 2) * 2.0 ** -24 * (np.abs(X) @ np.abs(Vf)) * scale + 2.0 ** -24 * np.abs(ref)
    assert np.all(np.abs(Y - ref) <= bound)


@pytest.mark.parametrize("n,m,decay,rel", [(20000, 64, 0.2, 1e-2), (50000, 256, 0.1, 3e-3), (4096, 100, 0.5, 1e-1)])
def test_pod_mixed(H, n, m, decay, rel):
    sig = 10.0 ** (-decay * np.arange(min(n, m)))
    X = _f32(synth.prescribed_spectrum(n, m, sig, seed=n + m))
    fro2 = float(np.sum(X * X))
    eps = rel * math.sqrt(fro2)
    ref = oracle.pod(X, eps)
    full_s, _, _, _ = oracle.svd(X)
    tails = oracle.tail_sums(full_s)
    N, s, Y, tail, st = H.hapod_pod(to_dev(X, dtype=torch.float32), eps, H.HAPOD_MIXED_TF32X3)
    assert rank_agrees(N, ref.N, tails, eps, rel_window=1e-2)
    s = s.cpu().numpy()
    k = min(N, ref.N)
    assert np.all(np.abs(s[:k] - ref.sigma[:k]) <= 10 * U_EFF * fro2 / ref.sigma[:k])
    assert projection_error(X, to_host(Y)) <= eps * eps * 1.01 + 10 * U_EFF * fro2 * 1e-3


def _u_eff(H, X, precision):
    """Measured Gram error of the form on X: ||G - G_ref||_2 / ||X||_F^2."""
    G = H.hapod_gram(to_dev(X, dtype=torch.float32), precision).cpu().numpy()
    ref = oracle.gram(X)
    return float(np.linalg.norm(G - ref, 2) / np.trace(ref))


@pytest.mark.parametrize("name,parent", [("star", synth.star_tree(6)), ("binary", synth.balanced_tree(2, 3)),
                                         ("chain", synth.chain_of_subtrees(3, 1))])
def test_hapod_mixed_trees(H, name, parent):
    rng = np.random.default_rng(len(parent))
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(20, 130))
    S = sum(cols)
    X = _f32(synth.advection_diffusion(1 << 15, S, seed=S))
    eps = 1e-2 * float(np.linalg.norm(X))
    _, data = leaf_split(X, parent, cols)
    ctx = H.hapod_create(parent, cols, eps, 0.5, X.shape[0], H.HAPOD_MIXED_TF32X3)
    bufs = {a: to_dev(data[a], dtype=torch.float32) for a in leaves}
    for a in leaves:
        H.hapod_push(ctx, a, bufs[a])
    s, U, st = H.hapod_result(ctx)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), 0.5)
    ref = oracle.hapod(parent, data, eps_nodes, keep_all=True)
    root = parent.index(-1)
    Uh = to_host(U)
    bound = sum(e * e for e in eps_nodes)
    assert projection_error(X, Uh) <= bound * 1.01
    assert abs(len(s) - ref[root].N) <= 1
    # CholQR2 at the root: orthonormal to FP32 working precision
    assert np.max(np.abs(Uh.T @ Uh - np.eye(Uh.shape[1]))) <= 1e-5
    # refreshed singular values, always checked on the common leading part: the
    # eigenvalue perturbation of each level's Gram error (u_eff measured on the leaves,
    # ||X||_F^2 bounding every node's trace) plus, where a node kept a different rank
    # than the oracle, the size of the extra mode (<= eps(a)) that entered its parent
    u_eff = max(_u_eff(H, data[a], H.HAPOD_MIXED_TF32X3) for a in leaves)
    levels = max(st_["level"] for st_ in stats)
    fro2 = float(np.sum(X * X))
    differ = [a for a in range(len(parent)) if a != root and stats[a]["k"] != ref[a].N]
    slack = math.sqrt(sum(eps_nodes[a] ** 2 for a in differ))
    sr = ref[root].sigma
    k = min(len(s), len(sr))
    dsig = np.abs(s.numpy()[:k] - sr[:k])
    assert np.all(dsig <= 10 * levels * u_eff * fro2 / sr[:k] + 1e-6 * sr[0] + slack), (dsig.max(), u_eff, differ)
