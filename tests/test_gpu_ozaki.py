"""Digit-slice FP64 form (HAPOD_FP64_OZAKI) on the GPU versus the CPU oracle.

The Gram is formed from an exact fixed-point representation of every column:
x = 2^E_j * (7 balanced base-256 digits), truncated below 2^(E_j - 55), with
2^E_j > max_i |x_ij|; digit pairs of level t + u <= 8 are summed exactly.  Per
row the product x_ri x_rj is then represented to within
2^(E_i + E_j) (2 * 2^-55 + 6.02 * 2^-56) < 1.26 * 2^(E_i + E_j - 53): the digit
truncation of both factors, plus the dropped levels t + u >= 9, dominated by the
six level-9 pairs of digits in [-128, 127] (at most 6 * 2^14 * 2^-72 of
2^(E_i + E_j + 2)), so

  |G_ij - G_ref_ij| <= 1.26 n 2^(E_i + E_j - 53) + 1e-13 sqrt(n) sqrt(G_ii G_jj)

the second term covering the rounding of the oracle's own FP64 sums and the
final FP64 rounding of the split sums.  Inputs whose digits are exact (small
integers) give the exact integer Gram, bit for bit.  The rest of the pipeline is
the FP64 form's, so the POD and HAPOD checks use the FP64 tolerances.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import leaf_split, projection_error, rank_agrees, sigma_close, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def col_exponents(X):
    """E_j with max_i |x_ij| < 2^E_j (frexp: m * 2^e, 0.5 <= m < 1); -1022 for zero columns."""
    mx = np.max(np.abs(X), axis=0) if X.shape[0] else np.zeros(X.shape[1])
    E = np.array([math.frexp(float(v))[1] if v > 0 else -1022 for v in mx])
    return np.maximum(E, -1022)


# worst-case representation error of one digit-slice product, in units of 2^(E_i + E_j - 53)
OZ_ROW = 1.26


def gram_bound(X, ref):
    n = X.shape[0]
    E = col_exponents(X)
    d = np.sqrt(np.abs(np.diag(ref)))
    return OZ_ROW * n * np.exp2(E[:, None] + E[None, :] - 53.0) + 1e-13 * math.sqrt(max(n, 1)) * np.outer(d, d)


@pytest.mark.parametrize("n,m,ld", [(1, 1, 1), (1000, 1, 1000), (10000, 100, 10000), (3000, 130, 3001),
                                    (50000, 7, 50000), (257, 64, 300), (70, 200, 70), (4100, 300, 4100),
                                    (200000, 20, 200001), (17, 129, 17)])
def test_gram_oz(H, n, m, ld):
    rng = np.random.default_rng(n + 3 * m)
    X = rng.standard_normal((n, m)) * (1.0 + np.arange(m))
    G = H.hapod_gram(to_dev(X, ld=ld), H.HAPOD_FP64_OZAKI).cpu().numpy()
    ref = oracle.gram(X)
    assert np.array_equal(G, G.T)
    err = np.abs(G - ref)
    bound = gram_bound(X, ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("n,m", [(5000, 40), (3001, 150), (20000, 9)])
def test_gram_oz_exact_integers(H, n, m):
    """Digits of small integers are exact and so is every level sum: the exact Gram."""
    rng = np.random.default_rng(m)
    Xi = rng.integers(-1000, 1001, size=(n, m))
    Gi = Xi.T.astype(np.int64) @ Xi.astype(np.int64)
    G = H.hapod_gram(to_dev(Xi.astype(np.float64)), H.HAPOD_FP64_OZAKI).cpu().numpy()
    assert np.array_equal(G, Gi.astype(np.float64))


def test_gram_oz_scales_zero_and_denormal_columns(H):
    """Column exponents from 2^-1070 (denormal) to 2^+300; a zero column; mixed signs."""
    rng = np.random.default_rng(11)
    n = 3000
    X = rng.standard_normal((n, 8))
    X[:, 0] *= 2.0 ** 300
    X[:, 1] *= 2.0 ** -300
    X[:, 2] = 0.0
    X[:, 3] = rng.standard_normal(n) * 2.0 ** -1060  # mostly denormal
    X[:, 4] = np.where(rng.random(n) < 0.5, -1.0, 1.0) * 2.0 ** rng.integers(-40, 40, size=n)
    X[:, 5] *= 1e-5
    G = H.hapod_gram(to_dev(X), H.HAPOD_FP64_OZAKI).cpu().numpy()
    ref = oracle.gram(X)
    assert np.all(G[2, :] == 0) and np.all(G[:, 2] == 0)
    # the bound with the exponents of each column, plus the oracle's own gradual
    # underflow: each of its n products below 2^-1022 is rounded to a multiple of 2^-1074
    err = np.abs(G - ref)
    bound = gram_bound(X, ref) + n * 2.0 ** -1074
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_gram_oz_nonfinite_column(H, bad):
    X = np.random.default_rng(1).standard_normal((500, 6))
    X[123, 4] = bad
    G = H.hapod_gram(to_dev(X), H.HAPOD_FP64_OZAKI).cpu().numpy()
    assert np.all(np.isnan(G[4, :])) and np.all(np.isnan(G[:, 4]))
    keep = [0, 1, 2, 3, 5]
    ref = oracle.gram(X[:, keep])
    sub = G[np.ix_(keep, keep)]
    assert np.all(np.abs(sub - ref) <= gram_bound(X[:, keep], ref))


def test_gram_oz_row_chunks(H, monkeypatch):
    """A 1 MiB digit workspace cuts the node into row chunks (a few per round)."""
    rng = np.random.default_rng(5)
    n, m = 20011, 130
    X = rng.standard_normal((n, m))
    ref = oracle.gram(X)
    monkeypatch.setenv("HAPOD_OZ_WORKSPACE_MB", "1")
    G = H.hapod_gram(to_dev(X), H.HAPOD_FP64_OZAKI).cpu().numpy()
    monkeypatch.delenv("HAPOD_OZ_WORKSPACE_MB")
    G2 = H.hapod_gram(to_dev(X), H.HAPOD_FP64_OZAKI).cpu().numpy()
    bound = gram_bound(X, ref)
    assert np.all(np.abs(G - ref) <= bound)
    assert np.all(np.abs(G2 - ref) <= bound)


def test_gram_oz_empty(H):
    """n = 0 rows: G = 0 (C ABI called directly: torch reports a null pointer for empty views)."""
    import ctypes

    buf = torch.ones((5, 4), dtype=torch.float64, device="cuda")
    G = torch.full((5, 5), 7.0, dtype=torch.float64, device="cuda")
    st = H._lib.hapod_gram(H.HAPOD_FP64_OZAKI, 0, 5, ctypes.c_void_p(buf.data_ptr()), 4,
                           ctypes.c_void_p(G.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == H.HAPOD_OK and torch.all(G == 0)


# ------------------------------------------------------------------ K4 X V
def modes_bound(X, V, scale):
    """Per entry: 1.26 m 2^(F_c - 53) (digit truncation of X and of the rescaled V plus the
    dropped levels, per term below 1.26 2^(F_c - 53)) + the FP64 rounding of the reference,
    times |scale_c|; F_c = max_j (E_j + e(V_jc)) with |V_jc| < 2^e(V_jc)."""
    m = X.shape[1]
    E = col_exponents(X)
    ev = np.where(V != 0, np.frexp(V)[1], -10 ** 6)
    F = np.max(E[:, None] + ev, axis=0)
    rn = np.sqrt(np.sum(X * X, axis=1))[:, None] * np.linalg.norm(V, axis=0)[None, :]
    return (OZ_ROW * m * np.exp2(F - 53.0)[None, :] + 1e-13 * math.sqrt(m) * rn) * np.abs(scale)[None, :]


@pytest.mark.parametrize("n,m,N", [(1, 3, 2), (1000, 100, 37), (4097, 130, 65), (300, 1, 1), (12345, 64, 64),
                                   (5000, 500, 20), (70001, 256, 19), (129, 40, 33)])
def test_modes_oz(H, n, m, N):
    rng = np.random.default_rng(n + m + N)
    X = rng.standard_normal((n, m)) * (1.0 + np.arange(m)) ** 0.5
    V = np.asfortranarray(rng.standard_normal((m, N)) / math.sqrt(m))
    scale = rng.uniform(0.5, 2.0, N)
    Y = to_host(H.hapod_modes(to_dev(X), to_dev(V), N, torch.from_numpy(scale).cuda(), H.HAPOD_FP64_OZAKI))
    ref = (X @ V) * scale
    err = np.abs(Y - ref)
    bound = modes_bound(X, V, scale)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_modes_oz_exact_integers(H):
    """Small-integer X and V: every digit and level sum is exact, so is X V."""
    rng = np.random.default_rng(3)
    X = rng.integers(-1000, 1001, size=(7000, 90)).astype(np.float64)
    V = np.asfortranarray(rng.integers(-100, 101, size=(90, 23)).astype(np.float64))
    Y = to_host(H.hapod_modes(to_dev(X), to_dev(V), 23, None, H.HAPOD_FP64_OZAKI))
    ref = (X.astype(np.int64) @ V.astype(np.int64)).astype(np.float64)
    assert np.array_equal(Y, ref)


def test_modes_oz_nonfinite(H):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((600, 12))
    X[5, 3] = float("inf")
    V = np.asfortranarray(rng.standard_normal((12, 4)))
    Y = to_host(H.hapod_modes(to_dev(X), to_dev(V), 4, None, H.HAPOD_FP64_OZAKI))
    assert np.all(np.isnan(Y))


def test_modes_oz_row_chunks_and_ld(H, monkeypatch):
    """1 MiB digit workspace (row chunks), padded leading dimensions of X, V and Y."""
    rng = np.random.default_rng(6)
    n, m, N = 30011, 130, 40
    X = rng.standard_normal((n, m))
    V = rng.standard_normal((m, N)) / math.sqrt(m)
    Vd = to_dev(V, ld=m + 3)
    monkeypatch.setenv("HAPOD_OZ_WORKSPACE_MB", "1")
    Y = to_host(H.hapod_modes(to_dev(X, ld=n + 5), Vd, N, None, H.HAPOD_FP64_OZAKI))
    monkeypatch.delenv("HAPOD_OZ_WORKSPACE_MB")
    ref = X @ V
    assert np.all(np.abs(Y - ref) <= modes_bound(X, V, np.ones(N)))


# ------------------------------------------------------------------ one node
@pytest.mark.parametrize("n,m,decay,rel", [(2000, 50, 0.2, 1e-4), (5000, 130, 0.08, 1e-6), (600, 300, 0.05, 1e-3),
                                           (128, 8, 1.0, 0.5)])
def test_pod_oz(H, n, m, decay, rel):
    sig = 10.0 ** (-decay * np.arange(min(n, m)))
    X = synth.prescribed_spectrum(n, m, sig, seed=n + m, noise=1e-13)
    eps = rel * float(np.linalg.norm(X))
    ref = oracle.pod(X, eps)
    full_s, _, _, _ = oracle.svd(X)
    tails = oracle.tail_sums(full_s)
    N, s, Y, tail, st = H.hapod_pod(to_dev(X), eps, H.HAPOD_FP64_OZAKI)
    assert rank_agrees(N, ref.N, tails, eps)
    ok, err = sigma_close(s.cpu().numpy(), ref.sigma, 1e-6, 1e-5)
    assert ok, err
    assert projection_error(X, to_host(Y)) <= eps * eps * (1 + 1e-6) + 1e-24 * float(np.sum(X * X))


# ------------------------------------------------------------------ HAPOD trees
def _run_tree(H, parent, cols, X, eps, omega, max_pending=0):
    leaves, data = leaf_split(X, parent, cols)
    ctx = H.hapod_create(parent, cols, eps, omega, X.shape[0], H.HAPOD_FP64_OZAKI, max_pending_leaves=max_pending)
    bufs = {a: to_dev(data[a]) for a in leaves}
    for a in leaves:
        H.hapod_push(ctx, a, bufs[a])
    s, U, st = H.hapod_result(ctx)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    return s.numpy(), to_host(U), st, stats, data


@pytest.mark.parametrize("name,parent", [("star", synth.star_tree(6)), ("binary", synth.balanced_tree(2, 3)),
                                         ("chain", synth.chain_of_subtrees(3, 1))])
def test_hapod_trees_oz(H, name, parent):
    rng = np.random.default_rng(len(parent))
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(5, 40))
    S = sum(cols)
    X = synth.prescribed_spectrum(3000, S, 10.0 ** (-0.12 * np.arange(min(S, 150))), seed=S, noise=1e-12)
    eps = 1e-5 * float(np.linalg.norm(X))
    s, U, st, stats, data = _run_tree(H, parent, cols, X, eps, 0.5)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), 0.5)
    ref = oracle.hapod(parent, data, eps_nodes, keep_all=True)
    root = parent.index(-1)
    assert all(stats[a]["k"] == ref[a].N for a in range(len(parent)))
    ok, err = sigma_close(s, ref[root].sigma, 1e-6, 1e-5)
    assert ok, err
    assert projection_error(X, U) <= sum(e * e for e in eps_nodes) * (1 + 1e-6) + 1e-22 * float(np.sum(X * X))


def test_hapod_c1_two_level_oz(H):
    """n = 10,000, 8 leaves x 100 columns, sigma_j = 10^(-j/20), noise 1e-10,
    eps = 1e-6 ||X||_F, omega = 0.5: ranks and sigma as the oracle."""
    parent, data, X = synth.star_prescribed()
    cols = [0] + [100] * 8
    S = X.shape[1]
    eps = 1e-6 * float(np.linalg.norm(X))
    s, U, st, stats, data = _run_tree(H, parent, cols, X, eps, 0.5)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), 0.5)
    ref = oracle.hapod(parent, data, eps_nodes, keep_all=True)
    assert all(stats[a]["k"] == ref[a].N for a in range(len(parent)))
    ok, err = sigma_close(s, ref[0].sigma, 1e-6, 1e-5)
    assert ok, err
    assert projection_error(X, U) / S <= (eps / math.sqrt(S)) ** 2


def test_hapod_streamed_advection_oz(H):
    """Advection-diffusion snapshots on a streamed chain (max_pending_leaves = 1)."""
    parent = synth.chain_of_subtrees(4, 2)
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = 16
    S = sum(cols)
    X = synth.advection_diffusion(4096, S, seed=5)
    eps = 1e-5 * float(np.linalg.norm(X))
    s, U, st, stats, data = _run_tree(H, parent, cols, X, eps, 0.5, max_pending=1)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), 0.5)
    assert projection_error(X, U) <= sum(e * e for e in eps_nodes) * (1 + 1e-6) + 1e-22 * float(np.sum(X * X))


def test_profile_steps_oz(H):
    """HAPOD_FLAG_PROFILE: the digit conversion (step 'digits') is accounted apart from
    the tensor-core Gram (step 'gram'), with the algorithmic volumes of the method."""
    parent = synth.star_tree(3)
    cols = [0, 20, 30, 25]
    n = 5000
    X = synth.prescribed_spectrum(n, 75, 10.0 ** (-0.1 * np.arange(75)), seed=4, noise=1e-12)
    leaves, data = leaf_split(X, parent, cols)
    ctx = H.hapod_create(parent, cols, 1e-4 * float(np.linalg.norm(X)), 0.5, n, H.HAPOD_FP64_OZAKI,
                         flags=H.HAPOD_FLAG_PROFILE)
    bufs = {a: to_dev(data[a]) for a in leaves}
    for a in leaves:
        H.hapod_push(ctx, a, bufs[a])
    H.hapod_result(ctx)
    prof = H.hapod_profile(ctx)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    ms = [s_["m"] for s_ in stats if s_["m"] > 0]
    assert prof["gram"]["ms"] > 0 and prof["digits"]["ms"] > 0 and prof["modes"]["ms"] > 0
    assert prof["gram"]["launches"] >= 2 * 2 and prof["digits"]["launches"] >= 2 * 2  # two batches
    assert prof["gram"]["flops"] == pytest.approx(sum(n * m * (m + 1) for m in ms))
    assert prof["digits"]["bytes"] == pytest.approx(sum(22.0 * n * m for m in ms))
