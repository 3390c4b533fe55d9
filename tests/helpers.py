"""Shared helpers for the GPU parity tests (host-side only)."""
import math

import numpy as np
import torch

U64 = 2.0 ** -53


def to_dev(X: np.ndarray, dtype=torch.float64, ld: int = None) -> torch.Tensor:
    """n x m column-major CUDA tensor with the values of X (optionally padded to ld)."""
    n, m = X.shape
    ld = ld or n
    buf = torch.zeros((m, ld), dtype=dtype, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype)
    return buf[:, :n].t()


def to_host(Y: torch.Tensor) -> np.ndarray:
    return np.asfortranarray(Y.double().cpu().numpy())


def rank_agrees(k_gpu: int, k_ref: int, tails_ref: np.ndarray, eps: float, rel_window: float = 1e-6) -> bool:
    """Equal ranks, or a genuine near-tie of the discarded tail at eps^2 (Def. truncated POD)."""
    if k_gpu == k_ref:
        return True
    if abs(k_gpu - k_ref) != 1:
        return False
    j = min(k_gpu, k_ref)
    return abs(tails_ref[j + 1] - eps * eps) <= rel_window * eps * eps or abs(tails_ref[j] - eps * eps) <= rel_window * eps * eps


def rank_within(k_gpu: int, tails_ref: np.ndarray, eps: float, delta: float) -> bool:
    """k_gpu is the truncation rank of Def. truncated POD for some tolerance whose square
    lies within delta of eps^2: tails_ref[k] <= eps^2 + delta and, unless k = 0,
    tails_ref[k - 1] > eps^2 - delta (tails_ref[j] = sum_{i >= j} sigma_i^2 of the oracle).
    delta is the form's perturbation of the tail sums (e.g. m ||G - G_ref||_2)."""
    e2 = eps * eps
    if k_gpu < 0 or k_gpu >= len(tails_ref):
        return False
    return tails_ref[k_gpu] <= e2 + delta and (k_gpu == 0 or tails_ref[k_gpu - 1] > e2 - delta)


def sigma_close(s_gpu: np.ndarray, s_ref: np.ndarray, rtol: float, floor_rel: float):
    """Relative agreement of singular values above floor_rel * sigma_max."""
    k = min(len(s_gpu), len(s_ref))
    big = s_ref[:k] >= floor_rel * s_ref[0]
    err = np.abs(s_gpu[:k][big] - s_ref[:k][big]) / s_ref[:k][big]
    return (err.max() if err.size else 0.0) <= rtol, (err.max() if err.size else 0.0)


def projection_error(X: np.ndarray, U: np.ndarray) -> float:
    """sum_s ||s - Q Q^T s||^2 for Q an orthonormal basis of span(U) (explicit residual)."""
    if U.shape[1] == 0:
        return float(np.sum(X * X))
    Q, _ = np.linalg.qr(U)
    R = X - Q @ (Q.T @ X)
    return float(np.sum(R * R))


def leaf_split(X: np.ndarray, parent, cols):
    leaves = [a for a in range(len(parent)) if a not in set(p for p in parent if p >= 0)]
    data, off = {}, 0
    for a in leaves:
        data[a] = np.asfortranarray(X[:, off:off + cols[a]])
        off += cols[a]
    return leaves, data


def max_angle_sin(U1: np.ndarray, U2: np.ndarray) -> float:
    """sin of the largest principal angle between span(U1) and span(U2) (both orthonormal):
    the 2-norm of the part of U1 outside span(U2).  (sqrt(1 - cos^2) from the singular
    values of U1^T U2 would turn an orthonormality defect d of the columns into an
    apparent angle of sqrt(2 d).)"""
    if U1.shape[1] == 0:
        return 0.0
    return float(np.linalg.norm(U1 - U2 @ (U2.T @ U1), 2))
