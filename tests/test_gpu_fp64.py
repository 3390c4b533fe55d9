"""FP64 form on the GPU versus the CPU oracle, through the C ABI.

Tolerances (FP64 form):
  * Gram: |G - G_ref| <= 1e-13 sqrt(n) sqrt(G_ii G_jj) (rounding of n-term FP64 sums
    in two summation orders, ~u sqrt(n) with a margin of ~100);
  * eigenvalues: |lambda - sigma(X)^2| <= 50 m u lambda_max (Weyl, with the Gram's
    own rounding and the Jacobi backward error);
  * singular values after truncation: relative 1e-6 for sigma >= 1e-5 sigma_max;
  * ranks: equal unless the oracle's tail is within 1e-6 relative of eps^2;
  * projection error of the GPU modes within Thm. hapod_bound (x (1 + 1e-6)).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1607_05210_gb300 import synth
from tests.helpers import (U64, leaf_split, max_angle_sin, projection_error, rank_agrees, sigma_close, to_dev,
                           to_host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


# ------------------------------------------------------------------ K1 Gram
@pytest.mark.parametrize("n,m,ld", [(1, 1, 1), (1000, 1, 1000), (10000, 100, 10000), (3000, 130, 3001),
                                    (50000, 7, 50000), (257, 64, 300), (70, 200, 70)])
def test_gram_f64(H, n, m, ld):
    rng = np.random.default_rng(n + m)
    X = rng.standard_normal((n, m)) * (1.0 + np.arange(m))
    G = H.hapod_gram(to_dev(X, ld=ld), H.HAPOD_FP64).cpu().numpy()
    ref = oracle.gram(X)
    d = np.sqrt(np.diag(ref))
    tol = 1e-13 * math.sqrt(n) * np.outer(d, d)
    assert np.all(np.abs(G - ref) <= tol)
    assert np.array_equal(G, G.T)


# ------------------------------------------------------------------ K2 eig
@pytest.mark.parametrize("rot", ["fp64", "double-float"])
@pytest.mark.parametrize("m", [1, 2, 17, 100, 130, 256, 600])
def test_eig_f64(H, m, rot):
    """FP64 rotations (the FP64 forms) and double-float rotations (the mixed forms, unit
    roundoff 2^-47): the Jacobi residual G V - V Lambda scales with the rotation unit;
    the eigenvalues are FP64 Rayleigh quotients (second order in the eigenvector
    error), so their bound is the FP64 one for both."""
    precision, u_rot = (H.HAPOD_FP64, U64) if rot == "fp64" else (H.HAPOD_MIXED_FX3, 2.0 ** -47)
    n = max(2 * m, 50)
    sig = 10.0 ** (-np.arange(min(m, 60)) / 10.0)
    X = synth.prescribed_spectrum(n, m, sig, seed=m)
    ref_s, _, ref_V, _ = oracle.svd(X)
    G = oracle.gram(X)
    lam, V, sweeps, st = H.hapod_eig(torch.from_numpy(G).cuda(), precision)
    assert st == H.HAPOD_OK
    lam = lam.cpu().numpy()
    V = to_host(V)
    lam_ref = np.zeros(m)
    lam_ref[:ref_s.size] = ref_s ** 2
    assert np.all(np.diff(lam) <= 0) and np.all(lam >= 0)
    assert np.max(np.abs(lam - lam_ref)) <= 50 * m * U64 * lam_ref[0]
    r = int(np.sum(lam > 0))  # numerical rank: columns beyond it are zero
    # the pivoted Cholesky stops once the trace of its Schur complement S is at most
    # m u trace(G); by Ky Fan the eigenvalues it leaves out sum to at most trace(S)
    trace = float(np.trace(G))
    assert lam_ref[r:].sum() <= 2 * m * U64 * trace + 50 * m * U64 * lam_ref[0]
    assert np.max(np.abs(V[:, :r].T @ V[:, :r] - np.eye(r))) <= 1e-12 * max(m, 10)
    assert np.all(V[:, r:] == 0)
    assert np.max(np.abs(G @ V - V * lam)) <= 50 * m * u_rot * lam_ref[0]
    # leading eigenvectors (well separated) match the oracle's right singular vectors
    r = min(10, m)
    assert max_angle_sin(V[:, :r], ref_V[:, :r]) <= 1e-9


def test_eig_zero_and_nonfinite(H):
    lam, V, sweeps, st = H.hapod_eig(torch.zeros((5, 5), dtype=torch.float64, device="cuda"))
    assert st == H.HAPOD_OK and sweeps == 0 and torch.all(lam == 0) and torch.all(V == 0)
    G = torch.eye(4, dtype=torch.float64, device="cuda")
    G[1, 1] = float("nan")
    with pytest.raises(H.HapodError) as e:
        H.hapod_eig(G)
    assert e.value.status == H.HAPOD_ERR_NONFINITE


# ------------------------------------------------------------------ K3 truncation
@pytest.mark.parametrize("m,rel", [(1, 0.5), (31, 1e-3), (32, 1e-3), (33, 1e-2), (100, 1e-6), (1000, 1e-4),
                                   (4096, 1e-8), (50, 10.0)])
def test_truncate(H, m, rel):
    rng = np.random.default_rng(m)
    lam = np.sort(rng.exponential(size=m) * 10.0 ** (-rng.uniform(0, 12, size=m)))[::-1].copy()
    s = np.sqrt(lam)
    tails = oracle.tail_sums(s)
    eps = rel * math.sqrt(tails[0])
    N, tail = H.hapod_truncate(torch.from_numpy(lam).cuda(), eps)
    Nref = int(np.argmax(tails <= eps * eps))
    assert rank_agrees(N, Nref, tails, eps)
    assert tail == pytest.approx(tails[N], rel=1e-12, abs=1e-300)


def test_truncate_inclusive_threshold(H):
    lam = torch.tensor([45.0, 5.0], dtype=torch.float64, device="cuda")
    assert H.hapod_truncate(lam, math.sqrt(5.0))[0] == 1
    assert H.hapod_truncate(lam, math.sqrt(50.0))[0] == 0
    assert H.hapod_truncate(lam, math.sqrt(4.99))[0] == 2
    assert H.hapod_truncate(lam, 0.0)[0] == 2


# ------------------------------------------------------------------ K4 modes
@pytest.mark.parametrize("n,m,N", [(1, 3, 2), (1000, 100, 37), (4097, 130, 65), (300, 1, 1), (12345, 64, 64)])
def test_modes_f64(H, n, m, N):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, m))
    V = np.asfortranarray(rng.standard_normal((m, N)))
    scale = rng.uniform(0.5, 2.0, N)
    Y = to_host(H.hapod_modes(to_dev(X), to_dev(V), N, torch.from_numpy(scale).cuda(), H.HAPOD_FP64))
    ref = (X @ V) * scale
    bound = 1e-13 * math.sqrt(m) * np.sqrt(np.sum(X * X, axis=1))[:, None] * np.linalg.norm(V, axis=0) * scale
    assert np.all(np.abs(Y - ref) <= bound)


# ------------------------------------------------------------------ one node
@pytest.mark.parametrize("n,m,decay,rel", [(2000, 50, 0.2, 1e-4), (5000, 130, 0.08, 1e-6), (600, 300, 0.05, 1e-3),
                                           (128, 8, 1.0, 0.5)])
def test_pod_f64(H, n, m, decay, rel):
    sig = 10.0 ** (-decay * np.arange(min(n, m)))
    X = synth.prescribed_spectrum(n, m, sig, seed=n + m, noise=1e-13)
    eps = rel * float(np.linalg.norm(X))
    ref = oracle.pod(X, eps)
    full_s, _, _, _ = oracle.svd(X)
    tails = oracle.tail_sums(full_s)
    N, s, Y, tail, st = H.hapod_pod(to_dev(X), eps, H.HAPOD_FP64)
    assert rank_agrees(N, ref.N, tails, eps)
    ok, err = sigma_close(s.cpu().numpy(), ref.sigma, 1e-6, 1e-5)
    assert ok, err
    Yh = to_host(Y)
    # ||X v_j|| vs sqrt(lambda_j): equal up to O(u sigma_0^2 / sigma_j^2) (cond(G) = cond(X)^2)
    sh = s.cpu().numpy()
    rtol = 1e-10 + 100 * U64 * (sh[0] / sh) ** 2 if N else 0
    assert np.all(np.abs(np.linalg.norm(Yh, axis=0) - sh) <= rtol * sh)
    assert projection_error(X, Yh) <= eps * eps * (1 + 1e-6) + 1e-24 * float(np.sum(X * X))


def test_pod_passthrough_and_empty(H):
    X = np.random.default_rng(0).standard_normal((40, 5))
    N, s, Y, tail, _ = H.hapod_pod(to_dev(X), 0.0)
    assert N == 5 and torch.all(s == 1) and np.array_equal(to_host(Y), X)
    N, s, Y, tail, _ = H.hapod_pod(to_dev(X), 2.0 * float(np.linalg.norm(X)))
    assert N == 0


# ------------------------------------------------------------------ HAPOD trees
def _run_tree(H, parent, cols, X, eps, omega, override=None, max_pending=0, precision=0, push_order=None):
    n = X.shape[0]
    leaves, data = leaf_split(X, parent, cols)
    ctx = H.hapod_create(parent, cols, eps, omega, n, precision, eps_override=override,
                         max_pending_leaves=max_pending)
    bufs = {a: to_dev(data[a], dtype=H.DTYPE[precision]) for a in leaves}
    for a in (push_order or leaves):
        H.hapod_push(ctx, a, bufs[a])
    s, U, st = H.hapod_result(ctx)
    stats = [H.hapod_node_stats(ctx, a) for a in range(len(parent))]
    H.hapod_destroy(ctx)
    return s.numpy(), to_host(U), st, stats, data


def _check_tree(H, parent, cols, X, eps_rel, omega, override=None, max_pending=0, push_order=None):
    S = X.shape[1]
    eps = eps_rel * float(np.linalg.norm(X))
    s, U, st, stats, data = _run_tree(H, parent, cols, X, eps, omega, override, max_pending, push_order=push_order)
    eps_nodes = oracle.tolerances(parent, cols, eps / math.sqrt(S), omega, override)
    np.testing.assert_allclose([st_["eps"] for st_ in stats], eps_nodes, rtol=1e-14)
    ref = oracle.hapod(parent, data, eps_nodes, keep_all=True)
    root = parent.index(-1)
    # per-node ranks (a rank change upstream makes later comparisons bound-wise only)
    same = True
    for a in range(len(parent)):
        if stats[a]["k"] != ref[a].N:
            same = False
    if same:
        ok, err = sigma_close(s, ref[root].sigma, 1e-6, 1e-5)
        assert ok, err
    bound = sum(e * e for e in eps_nodes)
    assert projection_error(X, U) <= bound * (1 + 1e-6) + 1e-22 * float(np.sum(X * X))
    return s, U, stats, ref, same


@pytest.mark.parametrize("name,parent", [("star", synth.star_tree(6)), ("binary", synth.balanced_tree(2, 3)),
                                         ("ternary", synth.balanced_tree(3, 2)),
                                         ("chain", synth.chain_of_subtrees(3, 1))])
@pytest.mark.parametrize("omega", [0.5, 0.95])
def test_hapod_trees_f64(H, name, parent, omega):
    rng = np.random.default_rng(len(parent))
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(5, 40))
    S = sum(cols)
    X = synth.prescribed_spectrum(3000, S, 10.0 ** (-0.12 * np.arange(min(S, 150))), seed=S, noise=1e-12)
    _, _, _, _, same = _check_tree(H, parent, cols, X, 1e-5, omega)
    assert same


def test_hapod_streamed_chain_f64(H):
    """Incremental HAPOD (Sec. 3.2, skinny tree) processed as leaves arrive."""
    parent = synth.chain_of_subtrees(4, 2)
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = 16
    S = sum(cols)
    X = synth.advection_diffusion(4096, S, seed=5)
    _check_tree(H, parent, cols, X, 1e-5, 0.5, max_pending=1)


def test_hapod_c1_two_level_f64(H):
    """n = 10,000, 8 leaves x 100 columns, sigma_j = 10^(-j/20), noise 1e-10,
    eps = 1e-6 ||X||_F, omega = 0.5: against the oracle and the global bounds."""
    parent, data, X = synth.star_prescribed()
    cols = [0] + [100] * 8
    s, U, stats, ref, same = _check_tree(H, parent, cols, X, 1e-6, 0.5)
    assert same
    S = X.shape[1]
    eps = 1e-6 * float(np.linalg.norm(X))
    direct = oracle.pod(X, 0.5 * eps)  # POD(S, sqrt|S| omega eps*)
    assert len(s) <= direct.N  # Thm. cor:hapod_bound mode bound
    assert projection_error(X, U) / S <= (eps / math.sqrt(S)) ** 2


def test_hapod_passthrough_leaves_equal_direct_pod(H):
    parent = synth.star_tree(4)
    cols = [0, 20, 20, 20, 20]
    X = synth.prescribed_spectrum(800, 80, 10.0 ** (-0.1 * np.arange(80)), seed=3)
    eps = 1e-4 * float(np.linalg.norm(X))
    ovr = [float("nan"), 0.0, 0.0, 0.0, 0.0]
    s, U, st, stats, _ = _run_tree(H, parent, cols, X, eps, 0.7, override=ovr)
    direct = oracle.pod(X, stats[0]["eps"])
    assert len(s) == direct.N
    ok, err = sigma_close(s, direct.sigma, 1e-6, 1e-5)
    assert ok, err


def test_hapod_edge_cases(H):
    # single node = plain POD
    X = synth.prescribed_spectrum(500, 30, 0.7 ** np.arange(30), seed=9)
    eps = 1e-3 * float(np.linalg.norm(X))
    s, U, st, stats, _ = _run_tree(H, [-1], [30], X, eps, 0.5)
    assert len(s) == oracle.pod(X, eps).N
    # tolerance above ||X||: nothing kept at the root
    parent = synth.star_tree(2)
    s, U, st, stats, _ = _run_tree(H, parent, [0, 15, 15], X, 10.0 * float(np.linalg.norm(X)), 0.5)
    assert len(s) == 0 and U.shape == (500, 0)
    # one-column leaves and an all-zero leaf
    parent = synth.star_tree(3)
    Z = np.concatenate([X[:, :1], np.zeros((500, 1)), X[:, 1:2]], axis=1)
    s, U, st, stats, _ = _run_tree(H, parent, [0, 1, 1, 1], Z, 1e-8, 0.5)
    assert stats[2]["k"] == 0 and len(s) == 2


def test_hapod_error_paths(H):
    parent = synth.star_tree(2)
    X = to_dev(np.ones((64, 4)))
    ctx = H.hapod_create(parent, [0, 2, 2], 1e-3, 0.5, 64)
    with pytest.raises(H.HapodError) as e:
        H.hapod_push(ctx, 0, X[:, :2])
    assert e.value.status == H.HAPOD_ERR_STATE
    with pytest.raises(H.HapodError) as e:
        H.hapod_push(ctx, 1, X[:, :3])
    assert e.value.status == H.HAPOD_ERR_INVALID
    with pytest.raises(H.HapodError) as e:
        H.hapod_result(ctx)
    assert e.value.status == H.HAPOD_ERR_STATE
    H.hapod_push(ctx, 1, X[:, :2])
    with pytest.raises(H.HapodError) as e:
        H.hapod_push(ctx, 1, X[:, :2])
    assert e.value.status == H.HAPOD_ERR_STATE
    H.hapod_destroy(ctx)
    # NaN input is reported, not hidden
    Xn = np.ones((64, 2))
    Xn[3, 1] = float("nan")
    ctx = H.hapod_create([-1], [2], 1e-3, 0.5, 64)
    with pytest.raises(H.HapodError) as e:
        H.hapod_push(ctx, 0, to_dev(Xn))
    assert e.value.status == H.HAPOD_ERR_NONFINITE
    H.hapod_destroy(ctx)
