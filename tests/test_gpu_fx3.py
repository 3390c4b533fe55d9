"""Mixed fixed-point form (FP32 snapshots; tcgen05 Gram from four balanced 8-bit
digits per value, fixed-point per column, integer-exact sums) versus the CPU FP64
oracle run on the same FP32 values.

Tolerances, derived from the arithmetic of gram_fx3.cu:
  * Gram: column j is represented as an integer multiple of 2^(E_j - 31) with
    |x - x~| <= 2^(E_j - 32), 2^(E_j - 1) <= M_j < 2^E_j (M the column maximum of
    |x|); the thirteen kept digit pairs (levels 2..6) leave out less than
    2^(E_i + E_j - 38.9) per row; the level sums 2..4 are exact integers, the FP32
    rounding of L'_5 = L_5 + 2^-8 L_6 (56 steps per 128-row group, each below
    2^-24 |L'_5| <= 2^-1 of its unit) adds less than 2^(E_i + E_j - 40) per row, and
    the int64 sums are exact.  Per row: |x_i x_j - p| <= (2^-31 + 2^-38.9 + 2^-40)
    2^(E_i + E_j) <= 2^-27 M_i M_j, so |G - G_ref| <= 2^-27 n M_i M_j + the oracle's
    FP64 rounding (1e-13 sqrt(n) sqrt(G_ii G_jj)).
  * exact case: small integers are represented exactly and every sum is an exact
    integer, so G equals the oracle's bit for bit.
  * the precision workload's leaf tolerance (eps = 1e-4 rel, quaternary tree of depth
    4): the tail beyond the oracle's rank moves by less than a tenth of eps(a)^2.
  * singular values, ranks and projection error: as for the other mixed forms, with
    u_eff measured, at eps = 1e-4 rel on trees of the precision workload.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import leaf_split, projection_error, rank_agrees, rank_within, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def _f32(X):
    return np.asfortranarray(np.asarray(X, dtype=np.float32).astype(np.float64))


def _gram(H, X, ld=None):
    return H.hapod_gram(to_dev(X, dtype=torch.float32, ld=ld), H.HAPOD_MIXED_FX3).cpu().numpy()


def _column_bound(X):
    """2^-27 n M_i M_j, M the column maxima of |x|."""
    M = np.max(np.abs(X), axis=0)
    return 2.0 ** -27 * X.shape[0] * np.outer(M, M)


@pytest.mark.parametrize("n,m,ld,kind", [(1000, 1, 1000, "gauss"), (10000, 100, 10000, "gauss"),
                                         (3000, 130, 3004, "gauss"), (50000, 256, 50000, "smooth"),
                                         (70, 200, 72, "gauss"), (200000, 300, 200000, "smooth"),
                                         (64, 128, 64, "gauss"), (131072, 128, 131072, "smooth"),
                                         (33, 129, 33, "gauss"), (5000, 127, 5001, "scaled"),
                                         (7000, 450, 7000, "gauss"), (4100, 65, 4100, "pulses")])
def test_gram_fx3(H, n, m, ld, kind):
    rng = np.random.default_rng(n + m)
    if kind == "gauss":
        X = rng.standard_normal((n, m)) * (1.0 + np.arange(m)) / m
    elif kind == "scaled":  # columns over 2^-100 .. 2^100: the result is FP64, nothing overflows
        X = rng.standard_normal((n, m)) * 2.0 ** rng.integers(-100, 100, m)
    elif kind == "pulses":
        X = synth.advection_pulses(n, m, seed=m)
    else:
        X = synth.advection_diffusion(n, m, seed=m)
    X = _f32(X)
    G = _gram(H, X, ld)
    ref = oracle.gram(X)
    d = np.sqrt(np.diag(ref))
    bound = _column_bound(X) + 1e-13 * math.sqrt(n) * np.outer(d, d)
    rel = np.abs(G - ref) / np.maximum(np.outer(d, d), 1e-300)
    print(f"gram fx3 n={n} m={m} {kind}: max {rel.max():.3e} rms {np.sqrt(np.mean(rel ** 2)):.3e}")
    assert np.all(np.abs(G - ref) <= bound)
    assert np.array_equal(G, G.T)


def test_gram_fx3_exact_integers(H):
    rng = np.random.default_rng(3)
    n, m = 70000, 200
    X = rng.integers(-8, 9, (n, m)).astype(np.float64)
    G = _gram(H, X)
    assert np.array_equal(G, oracle.gram(X))


def test_gram_fx3_zero_and_nonfinite_columns(H):
    X = np.ones((500, 9))
    X[:, 5] = 0.0
    X[300:, 6] = 0.0  # zero in some blocks only
    X[7, 3] = np.inf
    X[450, 8] = np.nan
    G = _gram(H, X)
    assert np.all(np.isnan(G[3])) and np.all(np.isnan(G[:, 8]))
    ok = [0, 1, 2, 4, 5, 6, 7]
    ref = oracle.gram(X[:, ok])
    assert np.array_equal(G[np.ix_(ok, ok)], ref)


def test_gram_fx3_resolves_precision_workload_leaf_tolerance(H):
    """A leaf of the precision workload (128 snapshots) at n = 2^16: the tail beyond
    the oracle's rank at the eps = 1e-4 rel quaternary tree's leaf tolerance
    (Thm. cor:hapod_bound: |S~_a| / |S| = 128 / 32768, L_T = 5, omega = 0.5) moves by
    less than a tenth of eps(a)^2."""
    n, m = 1 << 16, 128
    X = _f32(synth.advection_pulses(n, m, 11))
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
    assert abs(tail_gpu - tails_ref[k]) <= 0.1 * eps2


@pytest.mark.parametrize("n,m,decay,rel", [(20000, 64, 0.2, 1e-2), (50000, 256, 0.1, 3e-3), (4096, 100, 0.5, 1e-1),
                                           (30000, 120, 0.05, 1e-4), (30000, 200, 0.05, 1e-5)])
def test_pod_fx3(H, n, m, decay, rel):
    sig = 10.0 ** (-decay * np.arange(min(n, m)))
    X = _f32(synth.prescribed_spectrum(n, m, sig, seed=n + m, noise=1e-7))
    fro2 = float(np.sum(X * X))
    eps = rel * math.sqrt(fro2)
    ref = oracle.pod(X, eps)
    full_s, _, _, _ = oracle.svd(X)
    tails = oracle.tail_sums(full_s)
    G = _gram(H, X)
    u_eff = float(np.linalg.norm(G - oracle.gram(X), 2) / fro2)
    N, s, Y, tail, st = H.hapod_pod(to_dev(X, dtype=torch.float32), eps, H.HAPOD_MIXED_FX3)
    # each tail sum moves by at most m ||G - G_ref||_2 (Weyl per eigenvalue)
    assert rank_within(N, tails, eps, m * u_eff * fro2), (N, ref.N)
    s = s.cpu().numpy()
    k = min(N, ref.N)
    assert np.all(np.abs(s[:k] - ref.sigma[:k]) <= 10 * u_eff * fro2 / ref.sigma[:k] + 1e-6 * ref.sigma[0])
    assert projection_error(X, to_host(Y)) <= eps * eps * 1.01 + 10 * u_eff * fro2


@pytest.mark.parametrize("name,parent", [("star", synth.star_tree(6)), ("binary", synth.balanced_tree(2, 3)),
                                         ("chain", synth.chain_of_subtrees(3, 1)),
                                         ("quaternary", synth.balanced_tree(4, 2))])
def test_hapod_fx3_trees(H, name, parent):
    rng = np.random.default_rng(len(parent))
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(20, 130))
    S = sum(cols)
    X = _f32(synth.advection_pulses(1 << 15, S, S))
    eps = 1e-4 * float(np.linalg.norm(X))
    _, data = leaf_split(X, parent, cols)
    ctx = H.hapod_create(parent, cols, eps, 0.5, X.shape[0], H.HAPOD_MIXED_FX3)
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
    assert np.max(np.abs(Uh.T @ Uh - np.eye(Uh.shape[1]))) <= 1e-5
    for a in range(len(parent)):
        if stats[a]["k"] == ref[a].N:
            continue
        kids = [b for b in range(len(parent)) if parent[b] == a]
        Xa = data[a] if not kids else np.concatenate([ref[b].Y for b in kids], axis=1)
        full_s, _, _, _ = oracle.svd(Xa, want_vectors=False)
        ua = float(np.linalg.norm(_gram(H, Xa) - oracle.gram(Xa), 2))
        assert rank_within(stats[a]["k"], oracle.tail_sums(full_s), eps_nodes[a], Xa.shape[1] * ua), a
    # singular values on the common leading part: the eigenvalue perturbation of every
    # node's Gram error (Weyl: |d sigma| <= ||E_a||_2 / (2 sigma) at node a; measured on
    # the oracle's input of each node), times 10, plus, where a node kept a different
    # rank than the oracle, the size of the extra mode (<= eps(a)) that entered its parent
    def node_input(a):
        kids = [b for b in range(len(parent)) if parent[b] == a]
        return data[a] if not kids else _f32(np.concatenate([ref[b].Y for b in kids], axis=1))

    e_nodes = [float(np.linalg.norm(_gram(H, node_input(a)) - oracle.gram(node_input(a)), 2))
               for a in range(len(parent))]
    fro2 = float(np.sum(X * X))
    u_eff = sum(e_nodes) / fro2
    differ = [a for a in range(len(parent)) if a != root and stats[a]["k"] != ref[a].N]
    slack = math.sqrt(sum(eps_nodes[a] ** 2 for a in differ))
    sr = ref[root].sigma
    k = min(len(s), len(sr))
    dsig = np.abs(s.numpy()[:k] - sr[:k])
    print(f"{name}: k={len(s)} ref={len(sr)} u_eff={u_eff:.2e} max dsig/s0={dsig.max() / sr[0]:.2e} differ={differ}")
    assert np.all(dsig <= 10 * u_eff * fro2 / sr[:k] + 1e-6 * sr[0] + slack), (dsig.max(), u_eff, differ)


@pytest.mark.parametrize("n,m,N,ld", [(1000, 100, 37, 1000), (4097, 130, 20, 4100), (300, 1, 1, 300),
                                      (12345, 64, 64, 12345), (9999, 256, 70, 9999), (50000, 450, 130, 50000),
                                      (3000, 128, 128, 3000), (2000, 300, 257, 2001), (700, 2049, 40, 700),
                                      (600, 4500, 24, 600)])
def test_modes_fx3(H, n, m, N, ld):
    """Y = X V diag(s) from digit products: per column pair the representation of x on
    the grid 2^(E_j - 30) (error 2^(E_j - 31), times |V| < 2^(F_c - E_j)), of V on the
    grid 2^(F_c - E_j - 31) (error 2^(F_c - E_j - 32), times |x| <= 2^E_j) and the
    dropped digit pairs t + u >= 4 (3.008 2^(F_c - 31)) give at most 2^(F_c - 28.9) per
    product; with 2^F_c <= 4 max_j M_j |V_jc| (M_j = max_r |x_rj|) that is
    m 2^-26.9 max_j M_j |V_jc|.  D2 (the leading digit pair) is exact.  D3 (unit
    2^(F_c - 21) <= 2^-19 max_j M_j |V_jc|) is an FP32 sum of m per-column terms of at
    most 24737 (= 64 128 + 128 128 + 2^-8 (64 128 + 2 128 128) + 2^-16 (64 128 +
    3 128 128)) in 9 ceil(m / 16) accumulation steps; at 2^-22 of the running magnitude
    per step (a factor 4 over round-to-nearest) its error is at most
    9 ceil(m / 16) m 24737 2^-41 max_j M_j |V_jc|.  The last term, 2^-22 |X V|, covers
    the FP32 roundings of Y (the fused 256 D2 + D3, the product with the mode's FP32
    factor, the FP32 rounding of s itself).  Worst cases aside, the rounding of the
    D3 sum behaves like a random walk, so the RMS error over all entries stays within
    2^-20 of the RMS of |X| |V| |s|: a dropped digit pair of the 2^-8 level (relative
    size about 2^-16) fails that check."""
    rng = np.random.default_rng(n + m)
    X = _f32(rng.standard_normal((n, m)) * 2.0 ** rng.integers(-3, 4, m))
    V = np.asfortranarray(rng.standard_normal((m, N)))
    scale = rng.uniform(0.5, 2.0, N)
    Y = to_host(H.hapod_modes(to_dev(X, dtype=torch.float32, ld=ld), to_dev(V), N, torch.from_numpy(scale).cuda(),
                              H.HAPOD_MIXED_FX3))
    ref = (X @ V) * scale
    M = np.max(np.abs(X), axis=0)
    mv = np.max(M[:, None] * np.abs(V), axis=0)
    d3 = 9 * math.ceil(m / 16) * m * 24737 * 2.0 ** -41
    bound = ((m * 2.0 ** -26.9 + d3) * mv + 2.0 ** -22 * np.abs(X @ V)) * scale
    err = np.abs(Y - ref)
    absprod = (np.abs(X) @ np.abs(V)) * scale
    rms_ratio = math.sqrt(np.mean(err ** 2)) / math.sqrt(np.mean(absprod ** 2))
    print(f"modes fx3 n={n} m={m} N={N}: max err/bound {np.max(err / bound):.3e}, rms err/rms |X||V| "
          f"2^{math.log2(max(rms_ratio, 1e-300)):.1f}")
    assert np.all(err <= bound)
    assert rms_ratio <= 2.0 ** -20


@pytest.mark.parametrize("n,m,N", [(5000, 200, 50), (900, 4500, 20)])
def test_modes_fx3_exact_integers(H, n, m, N):
    """Small integers have a single nonzero digit each (D3 = 0), so D2 -- exact in
    every group, kept as int32 across groups -- gives X V exactly."""
    rng = np.random.default_rng(9)
    X = rng.integers(-8, 9, (n, m)).astype(np.float64)
    V = np.asfortranarray(rng.integers(-8, 9, (m, N)).astype(np.float64))
    Y = to_host(H.hapod_modes(to_dev(X, dtype=torch.float32), to_dev(V), N, None, H.HAPOD_MIXED_FX3))
    assert np.array_equal(Y, X @ V)
