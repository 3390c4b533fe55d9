"""Seeded synthetic inputs and tree builders (no POD arithmetic lives here).

Both the CUDA path and the CPU oracle consume what these functions return; this
module contains neither Gram, eigen-, truncation nor mode arithmetic.  The inputs
stand in for the paper's PDE snapshot data (Sec. 4), which is not available:

* ``prescribed_spectrum``: X = Q diag(s) W^T + noise * N(0, 1), Q and W with
  orthonormal columns drawn from the seed (QR of Gaussian matrices).
* ``star_prescribed``: the 10,000-row, 8 x 100-column, sigma_j = 10^(-j/20)
  two-level workload (shared Q, W of 200 columns, noise 1e-10).
* ``advection_diffusion``: u(x, t) = sum_{k=1..32} a_k exp(-nu k^2 t) sin(k (x - c t))
  on the periodic grid x_i = 2 pi i / n, a_k ~ N(0, k^-2), t_j ~ U[0, 1], nu = 1e-3,
  c = 1.  Expanded as X = B C with B = [sin(k x), cos(k x)] (n x 64) so that large
  matrices are produced by one matrix product on the device.
* ``pulse_workload`` / ``pulse_snapshots`` / ``advection_pulses``: the
  advection-diffusion snapshots plus 64 travelling Gaussian pulses
  sum_p A_p exp(-d(x, x_p + c t)^2 / (2 w^2)), w = 0.01, A_p = 1/p, centres
  x_p ~ U[0, 2 pi), d the periodic distance (the precision workload), with snapshot
  times from Philox4x32-10 (counter = global column index, key = seed) so that any
  column range (a leaf, a stream chunk) is reproducible on its own; host twin of
  the library's device generator ``hapod_synth_snapshots`` (FP64 arithmetic here,
  FP32 there).
* ``uneven_leaf_cols`` / ``uneven_decays`` / ``shared_basis`` / ``uneven_leaf``: the
  batched workload's leaves, X_l = Q[:, :r] diag(10^(-delta_l j)) W_l^T + noise with a
  shared orthonormal Q, per-leaf orthonormal W_l, m_l ~ U{16..512} columns and
  delta_l ~ U[1/40, 1/10] decades per index.
* tree builders returning parent arrays (root has parent -1).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Tuple

import numpy as np


# ------------------------------------------------------------------ trees
def star_tree(num_leaves: int) -> List[int]:
    """Root 0 with leaves 1..num_leaves (distributed HAPOD, Sec. 3.2)."""
    return [-1] + [0] * num_leaves


def balanced_tree(arity: int, edge_depth: int, num_leaves: Optional[int] = None) -> List[int]:
    """Balanced ``arity``-ary tree with ``arity**edge_depth`` leaf slots, the first
    ``num_leaves`` of them used (index order); inner nodes with no leaf below are
    removed.  Node 0 is the root; leaves are the last nodes."""
    slots = arity ** edge_depth
    if num_leaves is None:
        num_leaves = slots
    # build level by level from the root
    levels: List[List[int]] = [[0]]
    parent = [-1]
    for d in range(edge_depth):
        nxt = []
        for p in levels[-1]:
            for _ in range(arity):
                parent.append(p)
                nxt.append(len(parent) - 1)
        levels.append(nxt)
    leaves = levels[-1]
    used = set(leaves[:num_leaves])
    keep = [False] * len(parent)
    for a in used:
        b = a
        while b >= 0 and not keep[b]:
            keep[b] = True
            b = parent[b]
    remap = {}
    for a in range(len(parent)):
        if keep[a]:
            remap[a] = len(remap)
    return [(-1 if parent[a] < 0 else remap[parent[a]]) for a in range(len(parent)) if keep[a]]


def nary_tree(num_leaves: int, edge_depth: int) -> List[int]:
    """Tree-shape workload of Sec. 4.2: ``num_leaves`` blocks on the first leaf slots
    of a balanced n-ary tree of edge depth ``edge_depth``, n the smallest arity with
    n**edge_depth >= num_leaves (n = ceil(s^(1/depth)))."""
    arity = 1
    while arity ** edge_depth < num_leaves:
        arity += 1
    return balanced_tree(arity, edge_depth, num_leaves)


def chain_of_subtrees(num_subtrees: int, subtree_edge_depth: int) -> List[int]:
    """Left-deep incremental chain (Sec. 3.2, skinny tree) whose inputs are roots of
    balanced binary subtrees: alpha_1 = subtree_1 root, alpha_l = POD(alpha_{l-1} U
    subtree_l root).  Node 0 is the final chain node."""
    parent: List[int] = []

    def add(p):
        parent.append(p)
        return len(parent) - 1

    def subtree(p, depth):
        r = add(p)
        if depth > 0:
            subtree(r, depth - 1)
            subtree(r, depth - 1)
        return r

    if num_subtrees == 1:
        subtree(-1, subtree_edge_depth)
        return parent
    top = add(-1)
    cur = top
    for l in range(num_subtrees - 1, 0, -1):
        # cur = chain node alpha_{l+1}; children: alpha_l (or subtree_1 root) and subtree_{l+1}
        subtree(cur, subtree_edge_depth)
        if l == 1:
            subtree(cur, subtree_edge_depth)
        else:
            cur = add(cur)
    return parent


def leaves_of(parent: List[int]) -> List[int]:
    has_child = [False] * len(parent)
    for p in parent:
        if p >= 0:
            has_child[p] = True
    return [a for a in range(len(parent)) if not has_child[a]]


# ------------------------------------------------------- prescribed spectrum
def orthonormal(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    """n x k matrix with orthonormal columns (QR of a Gaussian matrix)."""
    q, r = np.linalg.qr(rng.standard_normal((n, k)))
    return q * np.sign(np.diag(r))


def prescribed_spectrum(n: int, m: int, sigma, seed: int, noise: float = 0.0,
                        dtype=np.float64) -> np.ndarray:
    """X = Q diag(sigma) W^T + noise * N(0,1), Q: n x r, W: m x r, r = len(sigma)."""
    rng = np.random.default_rng(seed)
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    Q = orthonormal(rng, n, r)
    W = orthonormal(rng, m, r)
    X = (Q * sigma) @ W.T
    if noise:
        X = X + noise * rng.standard_normal((n, m))
    return np.asfortranarray(X.astype(dtype))


def star_prescribed(seed: int = 1607, n: int = 10_000, leaves: int = 8, cols: int = 100,
                    rank: int = 200, noise: float = 1e-10) -> Tuple[List[int], Dict[int, np.ndarray], np.ndarray]:
    """Two-level FP64 workload: n rows, ``leaves`` x ``cols`` snapshots,
    sigma_j = 10^(-j/20), j < rank, shared Q (n x rank) and W (leaves*cols x rank)."""
    sig = 10.0 ** (-np.arange(rank) / 20.0)
    X = prescribed_spectrum(n, leaves * cols, sig, seed, noise)
    parent = star_tree(leaves)
    data = {1 + i: np.asfortranarray(X[:, i * cols:(i + 1) * cols]) for i in range(leaves)}
    return parent, data, X


# --------------------------------------------------- advection-diffusion snapshots
NUM_HARMONICS = 32


def advection_diffusion_coeffs(num_cols: int, seed: int, nu: float = 1e-3, c: float = 1.0) -> np.ndarray:
    """Coefficient matrix C (64 x num_cols): column j holds the coefficients of
    sin(k x) (rows 0..31) and cos(k x) (rows 32..63) of u(., t_j), from
    sin(k(x - c t)) = sin(kx) cos(kct) - cos(kx) sin(kct).  One trajectory: the a_k
    are drawn once per seed, the t_j uniformly on [0, 1]."""
    rng = np.random.default_rng(seed)
    k = np.arange(1, NUM_HARMONICS + 1, dtype=np.float64)
    a = rng.standard_normal(NUM_HARMONICS) / k
    t = rng.uniform(0.0, 1.0, num_cols)
    damp = a[:, None] * np.exp(-nu * (k[:, None] ** 2) * t[None, :])
    C = np.empty((2 * NUM_HARMONICS, num_cols))
    C[:NUM_HARMONICS] = damp * np.cos(k[:, None] * c * t[None, :])
    C[NUM_HARMONICS:] = -damp * np.sin(k[:, None] * c * t[None, :])
    return C


def fourier_basis(n: int) -> np.ndarray:
    """B (n x 64) = [sin(k x_i), cos(k x_i)], x_i = 2 pi i / n, argument reduced
    exactly as 2 pi ((k i) mod n) / n."""
    i = np.arange(n, dtype=np.int64)
    k = np.arange(1, NUM_HARMONICS + 1, dtype=np.int64)
    ang = 2.0 * math.pi * ((i[:, None] * k[None, :]) % n) / n
    return np.concatenate([np.sin(ang), np.cos(ang)], axis=1)


def advection_diffusion(n: int, num_cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Host version: X = B C (n x num_cols), column-major."""
    X = fourier_basis(n) @ advection_diffusion_coeffs(num_cols, seed)
    return np.asfortranarray(X.astype(dtype))


def advection_diffusion_device(n: int, num_cols: int, seed: int, dtype, device, col_offset: int = 0,
                               total_cols: Optional[int] = None, out=None):
    """Device version (torch): columns [col_offset, col_offset + num_cols) of the
    ``total_cols``-column trajectory, as a column-major n x num_cols tensor view
    (storage num_cols x n).  The product B C is formed in FP64 and rounded once."""
    import torch

    total = total_cols if total_cols is not None else num_cols
    C = advection_diffusion_coeffs(total, seed)[:, col_offset:col_offset + num_cols]
    B = torch.from_numpy(fourier_basis(n)).to(device)
    Ct = torch.from_numpy(np.ascontiguousarray(C.T)).to(device)  # num_cols x 64
    Xt = Ct @ B.T  # num_cols x n, row j = column j of X
    Xt = Xt.to(dtype)
    if out is not None:
        out.copy_(Xt)
        return out
    return Xt


# --------------------------------------------------- travelling pulses
NUM_PULSES = 64
PULSE_WIDTH = 0.01


# --------------------------------------------------- counter-based snapshot times
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(counter, key) -> np.ndarray:
    """Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of
    (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
    with the key bumped by the Weyl constants after each round.  ``counter``: 4 x N
    unsigned 32-bit words, ``key``: two words; returns 4 x N words."""
    c = [np.asarray(w, dtype=np.uint64) & 0xFFFFFFFF for w in counter]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    mask = np.uint64(0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(PHILOX_M0) * c[0]
        p1 = np.uint64(PHILOX_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
        k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
    return np.stack([w.astype(np.uint32) for w in c])


def philox_times(seed: int, col0: int, ncols: int) -> np.ndarray:
    """t_g = (w0 2^21 + (w1 >> 11)) 2^-53 for global columns g = col0 .. col0 + ncols - 1,
    (w0, w1) the first two words of Philox4x32-10 with counter (g mod 2^32, g div 2^32,
    0, 0) and key (seed mod 2^32, seed div 2^32)."""
    g = np.arange(col0, col0 + ncols, dtype=np.uint64)
    zero = np.zeros_like(g)
    w = philox4x32_10([g & np.uint64(0xFFFFFFFF), g >> np.uint64(32), zero, zero], (seed, seed >> 32))
    bits = (w[0].astype(np.uint64) << np.uint64(21)) | (w[1].astype(np.uint64) >> np.uint64(11))
    return bits.astype(np.float64) * 2.0 ** -53


def pulse_workload(seed: int, num_pulses: int = NUM_PULSES, nu: float = 1e-3, speed: float = 1.0,
                 width: float = PULSE_WIDTH) -> Dict:
    """Parameters of the travelling-pulse trajectory: harmonic amplitudes a_k ~ N(0, k^-2)
    from the seed's stream, pulse centres x_p ~ U[0, 2 pi) from stream seed + 1, pulse
    amplitudes A_p = 1/p (1/f decay), width w, nu, c, and the Philox key (the seed)."""
    rng = np.random.default_rng(seed)
    k = np.arange(1, NUM_HARMONICS + 1, dtype=np.float64)
    a = rng.standard_normal(NUM_HARMONICS) / k
    rng_p = np.random.default_rng(seed + 1)
    xp = rng_p.uniform(0.0, 2.0 * math.pi, NUM_PULSES)[:num_pulses]
    amp = 1.0 / np.arange(1, num_pulses + 1, dtype=np.float64)
    return {"seed": int(seed), "harmonic_amp": a, "nu": float(nu), "speed": float(speed),
            "pulse_centre": xp, "pulse_amp": amp, "pulse_width": float(width)}


def pulse_snapshots(n: int, col0: int, ncols: int, params: Dict, dtype=np.float32) -> np.ndarray:
    """Host twin of the device generator: columns col0 .. col0 + ncols - 1 (n x ncols,
    column-major), evaluated in FP64 and rounded once to ``dtype``."""
    t = philox_times(params["seed"], col0, ncols)
    k = np.arange(1, NUM_HARMONICS + 1, dtype=np.float64)
    damp = params["harmonic_amp"][:, None] * np.exp(-params["nu"] * (k[:, None] ** 2) * t[None, :])
    C = np.empty((2 * NUM_HARMONICS, ncols))
    C[:NUM_HARMONICS] = damp * np.cos(k[:, None] * params["speed"] * t[None, :])
    C[NUM_HARMONICS:] = -damp * np.sin(k[:, None] * params["speed"] * t[None, :])
    X = fourier_basis(n) @ C
    w = params["pulse_width"]
    h = 2.0 * math.pi / n
    R = int(math.ceil(9.0 * w / h)) + 1  # rows around the nearest grid point that can lie within 9 w
    off = np.arange(-R, R + 1)
    jj = np.broadcast_to(np.arange(ncols)[:, None], (ncols, off.size))
    for c, a in zip(params["pulse_centre"], params["pulse_amp"]):
        pos = np.mod(c + params["speed"] * t, 2.0 * math.pi)
        rows = np.mod(np.rint(pos / h).astype(np.int64)[:, None] + off[None, :], n)  # ncols x (2R + 1)
        d = np.abs(2.0 * math.pi * rows / n - pos[:, None])
        d = np.minimum(d, 2.0 * math.pi - d)
        v = np.where(d <= 9.0 * w, a * np.exp(-d * d / (2.0 * w * w)), 0.0)
        if 2 * R + 1 <= n:  # rows of one column are distinct
            X[rows, jj] += v
        else:
            np.add.at(X, (rows, jj), v)
    return np.asfortranarray(X.astype(dtype))


def advection_pulses(n: int, num_cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Columns 0 .. num_cols - 1 of the travelling-pulse trajectory of ``seed``."""
    return pulse_snapshots(n, 0, num_cols, pulse_workload(seed), dtype)


# --------------------------------------------------- uneven prescribed-spectrum leaves
def uneven_leaf_cols(seed: int, num_leaves: int, lo: int = 16, hi: int = 512) -> np.ndarray:
    """Column counts m_l ~ U{lo .. hi} of the batched workload's leaves."""
    return np.random.default_rng(seed).integers(lo, hi + 1, num_leaves)


def uneven_decays(seed: int, num_leaves: int, lo: float = 1.0 / 40.0, hi: float = 1.0 / 10.0) -> np.ndarray:
    """Per-leaf decay rates delta_l ~ U[lo, hi] decades per index (sigma_j = 10^(-delta_l j))."""
    return np.random.default_rng(seed + 1).uniform(lo, hi, num_leaves)


def shared_basis(seed: int, n: int, rank: int = 200) -> np.ndarray:
    """The leaves' shared left factor Q (n x rank, orthonormal columns)."""
    return orthonormal(np.random.default_rng(seed + 2), n, rank)


def leaf_factors(seed: int, leaf: int, m: int, rank: int, delta: float):
    """(W_l, sigma_l): W_l m x r orthonormal, sigma_j = 10^(-delta j), r = min(m, rank)."""
    r = min(m, rank)
    W = orthonormal(np.random.default_rng([seed, leaf]), m, r)
    return W, 10.0 ** (-delta * np.arange(r))


def uneven_leaf(Q: np.ndarray, seed: int, leaf: int, m: int, delta: float, noise: float = 1e-10,
                dtype=np.float64) -> np.ndarray:
    """Leaf l of the batched workload: Q[:, :r] diag(sigma_l) W_l^T + noise N(0, 1)
    (n x m, column-major), r = min(m, rank of Q)."""
    W, s = leaf_factors(seed, leaf, m, Q.shape[1], delta)
    X = (Q[:, :W.shape[1]] * s) @ W.T
    if noise:
        X = X + noise * np.random.default_rng([seed, leaf, 1]).standard_normal(X.shape)
    return np.asfortranarray(X.astype(dtype))
