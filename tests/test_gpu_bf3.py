"""Mixed split-BF16 form (FP32 snapshots; tcgen05 Gram from the exact three-piece
bf16 split x = b1 + b2 + b3, FP32 sweeps then FP64 sweeps in the eigensolver, FP64
truncation, CholQR2 at the root) versus the CPU FP64 oracle run on the same FP32
values.

Tolerances, derived from the arithmetic of gram_bf3.cu:
  * Gram, worst case: the six kept piece products represent x_i x_j to within
    2^-25 |x_i x_j| (dropped products b2 b3, b3 b2, b3 b3 and the split's remainder
    |r| <= 2^-27 |x|); the FP32 tensor-core accumulation truncates at each of the 24
    MMA steps of a 64-row segment, each off by at most 2^-23 of the running
    |sum|, which is at most sum_r |x_ri x_rj| over the segment (1 + 2^-7 with the
    small pieces); compensated segment sums and FP64 split sums add far less.  With
    Cauchy-Schwarz: |G - G_ref| <= (24 * 2^-23 + 2^-24) sqrt(G_ii G_jj).
  * Gram, exact case: values that are bf16 numbers whose 64-row sums of products are
    integers below 2^24 are added exactly, so G is bit-for-bit the oracle's.
  * the noise the Gram error puts on the truncation, which the worst case bounds
    far too loosely, is measured on snapshots of the precision workload (advection-
    diffusion plus travelling pulses) and must stay below a tenth of the leaf
    tolerance of that workload's tree (eps = 1e-4 rel, quaternary tree of depth 4).
  * singular values and ranks: as for the other mixed form, with u_eff measured.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import leaf_split, projection_error, rank_agrees, rank_within, to_dev, to_host

pytestmark = pytest.mark.gpu
GRAM_WORST = 24 * 2.0 ** -23 + 2.0 ** -24


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def _f32(X):
    return np.asfortranarray(np.asarray(X, dtype=np.float32).astype(np.float64))


def _gram(H, X, ld=None):
    return H.hapod_gram(to_dev(X, dtype=torch.float32, ld=ld), H.HAPOD_MIXED_BF16X3).cpu().numpy()


@pytest.mark.parametrize("n,m,ld,kind", [(1000, 1, 1000, "gauss"), (10000, 100, 10000, "gauss"),
                                         (3000, 130, 3004, "gauss"), (50000, 256, 50000, "smooth"),
                                         (70, 200, 72, "gauss"), (200000, 300, 200000, "smooth"),
                                         (64, 128, 64, "gauss"), (131072, 128, 131072, "smooth"),
                                         (33, 129, 33, "gauss"), (5000, 127, 5001, "scaled")])
def test_gram_bf3(H, n, m, ld, kind):
    rng = np.random.default_rng(n + m)
    if kind == "gauss":
        X = rng.standard_normal((n, m)) * (1.0 + np.arange(m)) / m
    elif kind == "scaled":  # columns over 2^-30 .. 2^30 (64-row sums of squares stay in the FP32 range)
        X = rng.standard_normal((n, m)) * 2.0 ** rng.integers(-30, 30, m)
    else:
        X = synth.advection_diffusion(n, m, seed=m)
    X = _f32(X)
    G = _gram(H, X, ld)
    ref = oracle.gram(X)
    d = np.sqrt(np.diag(ref))
    scale = np.outer(d, d)
    rel = np.abs(G - ref) / np.maximum(scale, 1e-300)
    print(f"gram bf16x3 n={n} m={m} {kind}: max {rel.max():.3e} rms {np.sqrt(np.mean(rel ** 2)):.3e}")
    assert np.all(np.abs(G - ref) <= GRAM_WORST * scale)
    assert np.array_equal(G, G.T)


def test_gram_bf3_exact_integers(H):
    rng = np.random.default_rng(3)
    n, m = 70000, 200
    X = rng.integers(-8, 9, (n, m)).astype(np.float64)  # bf16-exact; 64-row sums of products < 2^24
    G = _gram(H, X)
    assert np.array_equal(G, oracle.gram(X))


def test_gram_bf3_nonfinite(H):
    X = np.ones((500, 9))
    X[7, 3] = np.inf
    G = _gram(H, X)
    assert not np.all(np.isfinite(G[3]))
    assert np.all(np.isfinite(np.delete(np.delete(G, 3, 0), 3, 1)))


def _pulses(n, m, seed):
    """Snapshots of the precision workload: advection-diffusion plus 64 travelling
    Gaussian pulses (width 0.01, amplitudes 1/p, centres uniform)."""
    return synth.advection_pulses(n, m, seed)


def test_gram_bf3_tail_noise_within_derived_bound(H):
    """The form's floor on a leaf of the precision workload (128 snapshots, n = 2^16):
    the tail beyond the oracle's rank at 1e-4 rel moves by at most the worst-case Gram
    bound summed over the tail's dimensions (Weyl per eigenvalue).  The fixed-point
    form (test_gpu_fx3.py) is the one that resolves this workload's leaf tolerance."""
    n, m = 1 << 16, 128
    X = _f32(_pulses(n, m, 11))
    tr = float(np.sum(X * X))
    eps2 = tr * 1e-8 * 0.75 / 4
    G = _gram(H, X)
    lam_gpu = np.sort(np.linalg.eigvalsh(G))[::-1]
    s_ref, _, _, _ = oracle.svd(X)
    lam_ref = s_ref ** 2
    tails_ref = np.concatenate([np.cumsum(lam_ref[::-1])[::-1], [0.0]])
    k = int(np.argmax(tails_ref <= eps2))
    tail_gpu = float(np.sum(lam_gpu[k:]))
    print(f"k={k} tail_ref={tails_ref[k] / tr:.3e} tail_gpu={tail_gpu / tr:.3e} eps2={eps2 / tr:.3e} (of trace)")
    assert abs(tail_gpu - tails_ref[k]) <= (m - k) * GRAM_WORST * tr


@pytest.mark.parametrize("n,m,decay,rel", [(20000, 64, 0.2, 1e-2), (50000, 256, 0.1, 3e-3), (4096, 100, 0.5, 1e-1)])
def test_pod_bf3(H, n, m, decay, rel):
    sig = 10.0 ** (-decay * np.arange(min(n, m)))
    X = _f32(synth.prescribed_spectrum(n, m, sig, seed=n + m))
    fro2 = float(np.sum(X * X))
    eps = rel * math.sqrt(fro2)
    ref = oracle.pod(X, eps)
    full_s, _, _, _ = oracle.svd(X)
    tails = oracle.tail_sums(full_s)
    G = _gram(H, X)
    u_eff = float(np.linalg.norm(G - oracle.gram(X), 2) / fro2)
    N, s, Y, tail, st = H.hapod_pod(to_dev(X, dtype=torch.float32), eps, H.HAPOD_MIXED_BF16X3)
    # each tail sum moves by at most m ||G - G_ref||_2 (Weyl per eigenvalue)
    assert rank_within(N, tails, eps, m * u_eff * fro2), (N, ref.N)
    s = s.cpu().numpy()
    k = min(N, ref.N)
    # |d lambda| <= ||E||_2 (Weyl) -> |d sigma| <= u_eff ||X||_F^2 / sigma, with 10x for the eigensolver
    assert np.all(np.abs(s[:k] - ref.sigma[:k]) <= 10 * u_eff * fro2 / ref.sigma[:k] + 1e-6 * ref.sigma[0])
    assert projection_error(X, to_host(Y)) <= eps * eps * 1.01 + 10 * u_eff * fro2


@pytest.mark.parametrize("name,parent", [("star", synth.star_tree(6)), ("binary", synth.balanced_tree(2, 3)),
                                         ("chain", synth.chain_of_subtrees(3, 1)),
                                         ("quaternary", synth.balanced_tree(4, 2))])
def test_hapod_bf3_trees(H, name, parent):
    rng = np.random.default_rng(len(parent))
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(20, 130))
    S = sum(cols)
    X = _f32(_pulses(1 << 15, S, S))
    eps = 1e-2 * float(np.linalg.norm(X))  # a tolerance this form's Gram floor resolves
    _, data = leaf_split(X, parent, cols)
    ctx = H.hapod_create(parent, cols, eps, 0.5, X.shape[0], H.HAPOD_MIXED_BF16X3)
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
    # ranks of every node: equal, or a near-tie of the oracle's own tail at eps(a)^2
    for a in range(len(parent)):
        if stats[a]["k"] == ref[a].N:
            continue
        kids = [b for b in range(len(parent)) if parent[b] == a]
        Xa = data[a] if not kids else np.concatenate([ref[b].Y for b in kids], axis=1)
        full_s, _, _, _ = oracle.svd(Xa, want_vectors=False)
        ua = float(np.linalg.norm(_gram(H, Xa) - oracle.gram(Xa), 2))
        assert rank_within(stats[a]["k"], oracle.tail_sums(full_s), eps_nodes[a], Xa.shape[1] * ua), a
    # singular values on the common leading part: Gram error of each level (u_eff
    # measured on the leaves) plus, where a node kept a different rank, its extra mode
    u_eff = max(float(np.linalg.norm(_gram(H, data[a]) - oracle.gram(data[a]), 2) / np.sum(data[a] ** 2))
                for a in leaves)
    levels = max(st_["level"] for st_ in stats)
    fro2 = float(np.sum(X * X))
    differ = [a for a in range(len(parent)) if a != root and stats[a]["k"] != ref[a].N]
    slack = math.sqrt(sum(eps_nodes[a] ** 2 for a in differ))
    sr = ref[root].sigma
    k = min(len(s), len(sr))
    dsig = np.abs(s.numpy()[:k] - sr[:k])
    assert np.all(dsig <= 10 * levels * u_eff * fro2 / sr[:k] + 1e-6 * sr[0] + slack), (dsig.max(), u_eff, differ)
