"""Oracle: POD per node (C, FP64) and the HAPOD recursion over a rooted tree.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper references (arXiv 1607.05210):
  * Def. POD, Eq. snapshot_map (Sec. 2): singular values/modes of the snapshot map.
  * Def. truncated POD (Sec. 2): N = min{N' : sum_{n>N'} sigma_n^2 <= eps^2},
    POD(S, 0) = {(1, s)}.
  * Def. Rooted Tree (Sec. 3.1): children map, leaves, level
    L(a) = max(levels of children, 0) + 1, depth L_T = L(root).
  * Def. HAPOD (Sec. 3.1): HAPOD(a) = POD(S_a, eps(a)); leaf input D^-1(a);
    inner input = union over children of {sigma_n * phi_n}.
  * Thm. cor:hapod_bound (Sec. 3.3): eps(root) = sqrt|S| * omega * eps*,
    eps(a) = sqrt|S~_a| * (L_T - 1)^(-1/2) * sqrt(1 - omega^2) * eps*.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile hapod_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    src = os.path.join(_HERE, "hapod_oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        import subprocess

        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        i64, dp, d = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_double
        lib.oracle_gram.argtypes = [i64, i64, dp, i64, dp]
        lib.oracle_gram.restype = None
        lib.oracle_svd.argtypes = [i64, i64, dp, i64, dp, dp, dp]
        lib.oracle_svd.restype = ctypes.c_int
        lib.oracle_tail_sums.argtypes = [i64, dp, dp]
        lib.oracle_tail_sums.restype = None
        lib.oracle_pod.argtypes = [i64, i64, dp, i64, d, ctypes.POINTER(i64), dp, dp, dp]
        lib.oracle_pod.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_fortran64(X) -> np.ndarray:
    return np.asfortranarray(np.asarray(X, dtype=np.float64))


# --------------------------------------------------------------------------- POD
def gram(X) -> np.ndarray:
    """G = X^T X written as the plain sum (method of snapshots, Sec. 2 Remark)."""
    X = _as_fortran64(X)
    n, m = X.shape
    G = np.zeros((m, m), dtype=np.float64, order="F")
    _load().oracle_gram(n, m, _ptr(X), max(n, 1), _ptr(G))
    return G


def svd(X, want_vectors: bool = True):
    """Thin SVD of the snapshot map (Def. POD): Householder QR + one-sided Jacobi.

    Returns (sigma, US, V, sweeps): sigma descending (min(n, m) values), US = U diag(sigma)
    (n x r), V right singular vectors (m x r).
    """
    X = _as_fortran64(X)
    n, m = X.shape
    r = min(n, m)
    sigma = np.zeros(r)
    US = np.zeros((n, r), order="F") if want_vectors else None
    V = np.zeros((m, r), order="F") if want_vectors else None
    st = _load().oracle_svd(n, m, _ptr(X), max(n, 1), _ptr(sigma), _ptr(US), _ptr(V))
    if st == -2:
        raise MemoryError("oracle_svd: allocation failed")
    if st == -1:
        raise ArithmeticError("oracle_svd: one-sided Jacobi did not converge in 60 sweeps")
    return sigma, US, V, st


def tail_sums(sigma) -> np.ndarray:
    """tail[N'] = sum_{j >= N'} sigma_j^2 for N' = 0..r (Eq. pod_error)."""
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    out = np.zeros(s.size + 1)
    _load().oracle_tail_sums(s.size, _ptr(s), _ptr(out))
    return out


class PodResult:
    __slots__ = ("N", "sigma", "Y", "tail", "sweeps", "passthrough")

    def __init__(self, N, sigma, Y, tail, sweeps, passthrough):
        self.N, self.sigma, self.Y, self.tail = N, sigma, Y, tail
        self.sweeps, self.passthrough = sweeps, passthrough


def pod(X, eps: float) -> PodResult:
    """POD(S, eps) of Sec. 2 (Def. truncated POD); Y holds sigma_n * phi_n, n < N."""
    X = _as_fortran64(X)
    n, m = X.shape
    cap = m if eps == 0.0 else min(n, m)
    sigma = np.zeros(max(cap, 1))
    Y = np.zeros((n, max(cap, 1)), order="F")
    N = ctypes.c_int64(0)
    tail = ctypes.c_double(0.0)
    st = _load().oracle_pod(n, m, _ptr(X), max(n, 1), float(eps), ctypes.byref(N), _ptr(sigma), _ptr(Y),
                            ctypes.byref(tail))
    if st == -2:
        raise MemoryError("oracle_pod: allocation failed")
    if st == -1:
        raise ArithmeticError("oracle_pod: one-sided Jacobi did not converge in 60 sweeps")
    k = N.value
    return PodResult(k, sigma[:k].copy(), np.asfortranarray(Y[:, :k]), tail.value, st, eps == 0.0)


# ---------------------------------------------------------------------- tree / eps
def _children(parent: Sequence[int]) -> List[List[int]]:
    ch: List[List[int]] = [[] for _ in parent]
    for a, p in enumerate(parent):
        if p >= 0:
            ch[p].append(a)
    return ch


def _root(parent: Sequence[int]) -> int:
    roots = [a for a, p in enumerate(parent) if p < 0]
    if len(roots) != 1:
        raise ValueError("a rooted tree has exactly one root")
    return roots[0]


def _postorder(parent: Sequence[int]) -> List[int]:
    ch = _children(parent)
    out, stack = [], [(_root(parent), False)]
    while stack:
        a, done = stack.pop()
        if done:
            out.append(a)
            continue
        stack.append((a, True))
        for c in reversed(ch[a]):
            stack.append((c, False))
    if len(out) != len(parent):
        raise ValueError("tree is not connected to its root (Eq. treeconnected)")
    return out


def tree_levels(parent: Sequence[int]) -> List[int]:
    """L_T(a) = max({L_T(b) : b child of a} U {0}) + 1 (Def. Rooted Tree)."""
    ch = _children(parent)
    lev = [0] * len(parent)
    for a in _postorder(parent):
        lev[a] = max([lev[b] for b in ch[a]] + [0]) + 1
    return lev


def accumulated_counts(parent: Sequence[int], leaf_cols: Sequence[int]) -> List[int]:
    """|S~_a|: number of snapshots in the leaves below a (Thm. hapod_bound)."""
    ch = _children(parent)
    acc = [0] * len(parent)
    for a in _postorder(parent):
        acc[a] = int(leaf_cols[a]) if not ch[a] else sum(acc[b] for b in ch[a])
    return acc


def tolerances(parent: Sequence[int], leaf_cols: Sequence[int], eps_star: float, omega: float,
               override: Optional[Sequence[float]] = None) -> List[float]:
    """Local tolerances of Thm. cor:hapod_bound.

    eps(root) = sqrt(|S|) * omega * eps*;  eps(a) = sqrt(|S~_a|) * (L_T - 1)^(-1/2)
    * sqrt(1 - omega^2) * eps* for a != root.  A tree of depth 1 (a single node) has
    no non-root nodes; its root takes the whole budget, eps = sqrt(|S|) * eps*.
    ``override[a]`` (not NaN) replaces eps(a), e.g. 0 for a pass-through node.
    """
    lev = tree_levels(parent)
    acc = accumulated_counts(parent, leaf_cols)
    root = _root(parent)
    LT = lev[root]
    eps = [0.0] * len(parent)
    for a in range(len(parent)):
        if a == root:
            eps[a] = math.sqrt(acc[a]) * (omega if LT > 1 else 1.0) * eps_star
        else:
            eps[a] = math.sqrt(acc[a]) * (LT - 1) ** -0.5 * math.sqrt(max(0.0, 1.0 - omega * omega)) * eps_star
        if override is not None and not math.isnan(override[a]):
            eps[a] = float(override[a])
    return eps


# ------------------------------------------------------------------------- HAPOD
def hapod(parent: Sequence[int], leaf_data: Dict[int, np.ndarray], eps: Sequence[float],
          keep_all: bool = False):
    """HAPOD(root) by post-order recursion (Def. HAPOD).

    ``leaf_data[a]`` is the n x |D^-1(a)| snapshot matrix of leaf a.  The input of an
    inner node is the column concatenation of its children's outputs (in increasing
    node order).  Returns dict node -> PodResult (children are dropped once their
    parent is done unless ``keep_all``).
    """
    ch = _children(parent)
    out: Dict[int, PodResult] = {}
    for a in _postorder(parent):
        if ch[a]:
            X = np.concatenate([out[b].Y for b in ch[a]], axis=1)
        else:
            X = leaf_data[a]
        out[a] = pod(X, eps[a])
        if not keep_all:
            for b in ch[a]:
                out[b].Y = None
    return out


# ------------------------------------------------------------------ error measures
def projection_error(X, Q) -> float:
    """sum_s ||s - Q Q^T s||^2 with the residual formed explicitly (Thm. hapod_bound)."""
    X = np.asarray(X, dtype=np.float64)
    R = X - Q @ (Q.T @ X)
    return float(np.sum(R * R))
