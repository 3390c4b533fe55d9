"""Pins for the CPU FP64 oracle against things other than itself.

Each pin is chosen so that a plausible mistake in the oracle (dropped term, wrong
sign or index, transposed operand, off-by-one truncation) fails at least one test:
  * LAPACK SVD on tiny inputs (independent implementation) and exact reconstruction;
  * prescribed spectra and the hand-computed 2x2 example (tests/golden/);
  * invariances of singular values;
  * the Schmidt-Eckart-Young-Mirsky identity (Sec. 2, Eq. pod_error) with the
    residual formed explicitly, and the inclusive truncation rule (Def. truncated POD);
  * the advection-diffusion closed form (Fourier orthogonality on the periodic grid);
  * Thm. hapod_bound, Thm. mode_bound and Thm. cor:hapod_bound (Sec. 3.3) on
    random trees, and the special cases of Sec. 3.2 / Def. truncated POD.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1607_05210_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ------------------------------------------------------------------ SVD / POD
@pytest.mark.parametrize("n,m,rank", [(1, 1, 1), (5, 1, 1), (1, 5, 1), (30, 7, 7), (7, 30, 7), (64, 16, 16),
                                      (40, 16, 5), (16, 16, 16), (3, 9, 3)])
def test_svd_matches_lapack(n, m, rank):
    rng = np.random.default_rng(n * 100 + m)
    X = rng.standard_normal((n, rank)) @ rng.standard_normal((rank, m))
    s, US, V, sweeps = oracle.svd(X)
    ref = np.linalg.svd(X, compute_uv=False)
    assert sweeps >= 1
    np.testing.assert_allclose(s, ref, rtol=0, atol=1e-13 * ref[0])
    # exact reconstruction X = (U S) V^T over all min(n, m) triplets
    np.testing.assert_allclose(US @ V.T, X, rtol=0, atol=1e-13 * ref[0])
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-13)
    keep = s > 1e-10 * s[0]
    U = US[:, keep] / s[keep]
    np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-12)


def test_svd_golden_2x2():
    g = _golden()["svd_2x2"]
    s, _, _, _ = oracle.svd(np.array(g["X_rows"]))
    np.testing.assert_allclose(s, g["sigma"], rtol=1e-15)


@pytest.mark.parametrize("case", range(4))
def test_pod_inclusive_threshold_golden(case):
    g = _golden()["svd_2x2"]
    c = g["pod_cases"][case]
    r = oracle.pod(np.array(g["X_rows"]), math.sqrt(c["eps2"]))
    assert r.N == c["N"]


def test_prescribed_spectrum():
    sig = 10.0 ** (-np.arange(40) / 4.0)
    X = synth.prescribed_spectrum(300, 60, sig, seed=3)
    s, _, _, _ = oracle.svd(X)
    np.testing.assert_allclose(s[:40], sig, rtol=0, atol=2e-15 * 60)
    assert np.all(s[40:] <= 1e-14)
    # relative accuracy of the QR + one-sided Jacobi route down to 1e-7 of sigma_max
    big = sig > 1e-7
    np.testing.assert_allclose(s[:40][big], sig[big], rtol=1e-6)


def test_singular_value_invariances():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((50, 12)) * (2.0 ** np.arange(12))
    s0, _, _, _ = oracle.svd(X)
    Q = synth.orthonormal(rng, 50, 50)
    s1, _, _, _ = oracle.svd(Q @ X)
    s2, _, _, _ = oracle.svd(X[:, rng.permutation(12)])
    s3, _, _, _ = oracle.svd(-3.0 * X)
    np.testing.assert_allclose(s1, s0, rtol=1e-13)
    np.testing.assert_allclose(s2, s0, rtol=1e-13)
    np.testing.assert_allclose(s3, 3.0 * s0, rtol=1e-13)


def test_tail_sums_geometric_closed_form():
    q = 0.5
    s = q ** np.arange(30)  # sigma_j^2 = q^(2j): tail(N') = q^(2N') (1 - q^(2(30-N'))) / (1 - q^2)
    tail = oracle.tail_sums(s)
    Np = np.arange(31)
    ref = q ** (2 * Np) * (1 - q ** (2 * (30 - Np))) / (1 - q * q)
    np.testing.assert_allclose(tail, ref, rtol=1e-15, atol=0)


@pytest.mark.parametrize("rel", [0.3, 1e-2, 1e-4, 1e-7])
def test_pod_truncation_and_error_identity(rel):
    """N is minimal with tail <= eps^2 (Def. truncated POD) and the explicit residual
    equals the tail of sigma^2 (Eq. pod_error)."""
    sig = 10.0 ** (-np.arange(25) / 5.0)
    X = synth.prescribed_spectrum(200, 25, sig, seed=5)
    fro2 = float(np.sum(X * X))
    eps = rel * math.sqrt(fro2)
    r = oracle.pod(X, eps)
    s, _, _, _ = oracle.svd(X)
    tail = oracle.tail_sums(s)
    assert tail[r.N] <= eps * eps
    assert r.N == 0 or tail[r.N - 1] > eps * eps
    assert r.tail == pytest.approx(tail[r.N], rel=1e-12, abs=1e-300)
    # Y = U_N Sigma_N: columns orthogonal with norms sigma
    np.testing.assert_allclose(np.linalg.norm(r.Y, axis=0), r.sigma, rtol=1e-12)
    if r.N:
        Q = r.Y / r.sigma
        err = oracle.projection_error(X, Q)
        assert err == pytest.approx(r.tail, rel=1e-6, abs=1e-28 * fro2)
        assert err <= eps * eps * (1 + 1e-9)


def test_pod_eps_zero_is_passthrough():
    X = np.asfortranarray(np.random.default_rng(2).standard_normal((17, 6)))
    r = oracle.pod(X, 0.0)
    assert r.N == 6 and r.passthrough
    assert np.array_equal(r.Y, X)
    assert np.array_equal(r.sigma, np.ones(6))


def test_pod_eps_above_norm_keeps_nothing():
    X = np.random.default_rng(4).standard_normal((17, 6))
    r = oracle.pod(X, 1.0001 * np.linalg.norm(X))
    assert r.N == 0 and r.Y.shape == (17, 0)


def test_pod_zero_matrix():
    r = oracle.pod(np.zeros((20, 5)), 1e-3)
    assert r.N == 0 and r.tail == 0.0


def test_gram_definition():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((123, 9))
    G = oracle.gram(X)
    np.testing.assert_allclose(G, X.T @ X, rtol=1e-13, atol=1e-12)
    assert np.array_equal(G, G.T)


def test_advection_diffusion_closed_form():
    """Columns lie in span{sin kx, cos kx}, k=1..32, orthogonal on the periodic grid
    with squared norm n/2, so sigma(X) = sqrt(n/2) * sigma(C)."""
    n, cols = 2048, 96
    C = synth.advection_diffusion_coeffs(cols, seed=9)
    X = synth.advection_diffusion(n, cols, seed=9)
    s, _, _, _ = oracle.svd(X)
    ref = math.sqrt(n / 2) * np.linalg.svd(C, compute_uv=False)
    big = ref > 1e-9 * ref[0]
    np.testing.assert_allclose(s[:ref.size][big], ref[big], rtol=1e-7)
    assert np.all(s[ref.size:] <= 1e-12 * s[0])


# ------------------------------------------------------------------ tree / eps
@pytest.mark.parametrize("i", range(3))
def test_tolerances_golden(i):
    t = _golden()["trees"][i]
    assert oracle.tree_levels(t["parent"]) == t["levels"]
    assert oracle.accumulated_counts(t["parent"], t["leaf_cols"]) == t["acc"]
    eps = oracle.tolerances(t["parent"], t["leaf_cols"], t["eps_star"], t["omega"])
    np.testing.assert_allclose(eps, t["eps"], rtol=1e-14)


def _trees():
    return {
        "star8": synth.star_tree(8),
        "binary6": synth.balanced_tree(2, 6),
        "quaternary1000": synth.balanced_tree(4, 5, 1000),
        "chain4x4": synth.chain_of_subtrees(4, 4),
        "single": [-1],
    }


@pytest.mark.parametrize("name", list(_trees()))
@pytest.mark.parametrize("omega", [0.0, 0.5, 0.95, 1.0])
def test_tolerance_split_sums_to_budget(name, omega):
    """Proof of Thm. cor:hapod_bound: sum_gamma eps(gamma)^2 <= |S| eps*^2, using
    sum over each level of |S~_gamma| <= |S|."""
    parent = _trees()[name]
    rng = np.random.default_rng(len(parent))
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(1, 50))
    S = sum(cols)
    lev = oracle.tree_levels(parent)
    acc = oracle.accumulated_counts(parent, cols)
    for l in range(1, max(lev) + 1):
        assert sum(acc[a] for a in range(len(parent)) if lev[a] == l) <= S
    eps = oracle.tolerances(parent, cols, 0.01, omega)
    assert sum(e * e for e in eps) <= S * 1e-4 * (1 + 1e-12)


def test_tolerance_override():
    parent = synth.star_tree(3)
    eps = oracle.tolerances(parent, [0, 4, 4, 4], 0.1, 0.5, override=[float("nan"), 0.0, float("nan"), 0.25])
    assert eps[1] == 0.0 and eps[3] == 0.25 and eps[0] == pytest.approx(math.sqrt(12) * 0.05)


# ------------------------------------------------------------------ HAPOD theorems
def _random_case(parent, n, seed, decay=0.35, noise=1e-9):
    rng = np.random.default_rng(seed)
    leaves = synth.leaves_of(parent)
    cols = [0] * len(parent)
    for a in leaves:
        cols[a] = int(rng.integers(3, 14))
    S = sum(cols)
    sig = 10.0 ** (-decay * np.arange(min(n, S)))
    X = synth.prescribed_spectrum(n, S, sig, seed=seed + 1, noise=noise)
    data, off = {}, 0
    for a in leaves:
        data[a] = np.asfortranarray(X[:, off:off + cols[a]])
        off += cols[a]
    return cols, data, X


def _below(parent, a):
    ch = [[] for _ in parent]
    for b, p in enumerate(parent):
        if p >= 0:
            ch[p].append(b)
    out, st = [], [a]
    while st:
        b = st.pop()
        out.append(b)
        st.extend(ch[b])
    return out


TREES_SMALL = {
    "star": synth.star_tree(5),
    "binary": synth.balanced_tree(2, 3),
    "ternary": synth.balanced_tree(3, 2),
    "chain": synth.chain_of_subtrees(3, 1),
}


@pytest.mark.parametrize("name", list(TREES_SMALL))
@pytest.mark.parametrize("omega", [0.3, 0.9])
def test_hapod_error_and_mode_bounds(name, omega):
    """Thm. hapod_bound and Thm. mode_bound at every node, Thm. cor:hapod_bound globally."""
    parent = TREES_SMALL[name]
    cols, data, X = _random_case(parent, 120, seed=len(parent) * 7 + int(omega * 10))
    S = X.shape[1]
    eps_star = 1e-3 * math.sqrt(float(np.sum(X * X)) / S)
    eps = oracle.tolerances(parent, cols, eps_star, omega)
    res = oracle.hapod(parent, data, eps, keep_all=True)
    leaves = synth.leaves_of(parent)
    order = {a: i for i, a in enumerate(leaves)}
    offs = np.cumsum([0] + [cols[a] for a in leaves])
    for a in range(len(parent)):
        below = _below(parent, a)
        lv = sorted((b for b in below if b in order), key=lambda b: order[b])
        Xa = np.concatenate([X[:, offs[order[b]]:offs[order[b]] + cols[b]] for b in lv], axis=1)
        bound = sum(eps[g] ** 2 for g in below)
        Q = res[a].Y / res[a].sigma if res[a].N else np.zeros((X.shape[0], 0))
        err = oracle.projection_error(Xa, Q)
        assert err <= bound * (1 + 1e-8) + 1e-28, (a, err, bound)
        assert res[a].N <= oracle.pod(Xa, eps[a]).N
    root = [a for a, p in enumerate(parent) if p < 0][0]
    Q = res[root].Y / res[root].sigma
    assert oracle.projection_error(X, Q) / S <= eps_star ** 2 * (1 + 1e-8)
    assert res[root].N <= oracle.pod(X, math.sqrt(S) * omega * eps_star).N


def test_star_with_passthrough_leaves_equals_direct_pod():
    """Sec. 3.2 with eps(leaves) = 0 (Def. truncated POD, POD(S, 0)): the root sees S."""
    parent = synth.star_tree(4)
    cols, data, X = _random_case(parent, 80, seed=21)
    eps = oracle.tolerances(parent, cols, 1e-4, 0.7, override=[float("nan")] + [0.0] * 4)
    res = oracle.hapod(parent, data, eps)
    direct = oracle.pod(X, eps[0])
    assert res[0].N == direct.N
    np.testing.assert_array_equal(res[0].sigma, direct.sigma)


def test_single_node_tree_equals_pod():
    X = synth.prescribed_spectrum(60, 11, 0.5 ** np.arange(11), seed=2)
    eps = oracle.tolerances([-1], [11], 1e-3, 0.5)
    res = oracle.hapod([-1], {0: X}, eps)
    direct = oracle.pod(X, math.sqrt(11) * 1e-3)
    assert res[0].N == direct.N
    np.testing.assert_array_equal(res[0].sigma, direct.sigma)


# ------------------------------------------------------------------ planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """A truncation that keeps one mode too few, or a tolerance split without the
    (L_T - 1)^(-1/2) factor, must violate a pin above."""
    parent = synth.balanced_tree(2, 3)
    cols, data, X = _random_case(parent, 120, seed=77)
    S = X.shape[1]
    eps_star = 1e-3 * math.sqrt(float(np.sum(X * X)) / S)
    # (1) split without the level factor breaks the budget of Thm. cor:hapod_bound
    eps = oracle.tolerances(parent, cols, eps_star, 0.5)
    LT = max(oracle.tree_levels(parent))
    wrong = [e * math.sqrt(LT - 1) if p >= 0 else e for e, p in zip(eps, parent)]
    assert sum(e * e for e in wrong) > S * eps_star ** 2
    # (2) dropping one kept mode breaks Thm. hapod_bound at the root
    real_pod = oracle.core.pod

    def short_pod(Xa, e):
        r = real_pod(Xa, e)
        if r.N > 0 and e > 0:
            r.N -= 1
            r.sigma = r.sigma[:-1]
            r.Y = r.Y[:, :-1]
        return r

    monkeypatch.setattr(oracle.core, "pod", short_pod)
    res = oracle.hapod(parent, data, eps, keep_all=True)
    Q = res[0].Y / res[0].sigma
    assert oracle.projection_error(X, Q) > sum(e * e for e in eps)
