"""Thin Python binding of the C ABI in include/hapod.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Device buffers are
torch CUDA tensors (PyTorch is used for device memory and streams only); every
step of the computation runs in libhapod's CUDA kernels.  Loading fails loudly if
the library has not been built (``__graft_entry__.build()``): there is no CPU
fallback.

Matrices are column-major: an n x m snapshot matrix is passed as a tensor ``Xt``
of shape (m, n) (row j = snapshot j, contiguous) or as any tensor whose
transpose view is column-major; helpers below accept the (n, m) view with
``stride(0) == 1``.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence, Tuple

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhapod.so")

HAPOD_OK = 0
HAPOD_ERR_INVALID = 1
HAPOD_ERR_TREE = 2
HAPOD_ERR_STATE = 3
HAPOD_ERR_CUDA = 4
HAPOD_ERR_OOM = 5
HAPOD_ERR_NONFINITE = 6
HAPOD_ERR_TIMEOUT = 7
HAPOD_WARN_NOCONVERGE = 8
HAPOD_WARN_BELOW_FLOOR = 9
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_TREE", 3: "ERR_STATE", 4: "ERR_CUDA", 5: "ERR_OOM",
                6: "ERR_NONFINITE", 7: "ERR_TIMEOUT", 8: "WARN_NOCONVERGE", 9: "WARN_BELOW_FLOOR"}

HAPOD_FP64 = 0
HAPOD_MIXED_TF32X3 = 1
HAPOD_FP64_OZAKI = 2
HAPOD_MIXED_BF16X3 = 3
HAPOD_MIXED_FX3 = 4
DTYPE = {HAPOD_FP64: torch.float64, HAPOD_MIXED_TF32X3: torch.float32, HAPOD_FP64_OZAKI: torch.float64,
         HAPOD_MIXED_BF16X3: torch.float32, HAPOD_MIXED_FX3: torch.float32}


class hapod_tree(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_int32), ("parent", ctypes.POINTER(ctypes.c_int32)),
                ("leaf_cols", ctypes.POINTER(ctypes.c_int64))]


class hapod_tol(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("omega", ctypes.c_double),
                ("eps_override", ctypes.POINTER(ctypes.c_double)), ("precision", ctypes.c_int32),
                ("max_pending_leaves", ctypes.c_int32), ("flags", ctypes.c_int32)]


HAPOD_FLAG_PROFILE = 1
HAPOD_FLAG_RIGHT_VECTORS = 2
PROFILE_STEPS = ("gram", "eig", "truncate", "gather", "modes", "copy", "digits")


class hapod_profile_info(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8), ("bytes", ctypes.c_double * 8),
                ("flops", ctypes.c_double * 8)]


class hapod_node_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("k", ctypes.c_int64), ("eps", ctypes.c_double), ("tail_sq", ctypes.c_double),
                ("level", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("state", ctypes.c_int32),
                ("status", ctypes.c_int32)]


SYNTH_MAX_PULSES = 64


class hapod_synth_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("nu", ctypes.c_double), ("speed", ctypes.c_double),
                ("harmonic_amp", ctypes.c_double * 32), ("num_pulses", ctypes.c_int32),
                ("pulse_width", ctypes.c_double), ("pulse_centre", ctypes.c_double * SYNTH_MAX_PULSES),
                ("pulse_amp", ctypes.c_double * SYNTH_MAX_PULSES)]


class HapodError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhapod.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pi64, pd, pi32 = ctypes.POINTER(i64), ctypes.POINTER(d), ctypes.POINTER(i32)
    sig = {
        "hapod_create": ([ctypes.POINTER(hapod_tree), ctypes.POINTER(hapod_tol), i64, vp, ctypes.POINTER(vp)], i32),
        "hapod_push": ([vp, i32, vp, i64, i64], i32),
        "hapod_result": ([vp, pi64, pd, vp, i64], i32),
        "hapod_node_stats": ([vp, i32, ctypes.POINTER(hapod_node_info)], i32),
        "hapod_profile": ([vp, ctypes.POINTER(hapod_profile_info)], i32),
        "hapod_last_error": ([vp], ctypes.c_char_p),
        "hapod_destroy": ([vp], None),
        "hapod_trim_pool": ([vp], i32),
        "hapod_gram": ([i32, i64, i64, vp, i64, vp, vp], i32),
        "hapod_eig": ([i32, i64, vp, vp, vp, pi32, vp], i32),
        "hapod_truncate": ([i64, vp, d, pi64, pd, vp], i32),
        "hapod_modes": ([i32, i64, i64, vp, i64, vp, i64, i64, vp, vp, i64, vp], i32),
        "hapod_pod": ([i32, i64, i64, vp, i64, d, pi64, vp, vp, i64, pd, vp], i32),
        "hapod_gram_noalloc": ([i64, i64, vp, i64, vp, vp], i32),
        "hapod_result_right": ([vp, vp, i64], i32),
        "hapod_autotune": ([i32, i64, i64, vp, i64, ctypes.POINTER(i32), pd, vp], i32),
        "hapod_autotune_clear": ([], None),
        "hapod_synth_snapshots": ([ctypes.POINTER(hapod_synth_params), i64, i64, i64, i32, vp, i64, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()
EXPORTED = ("hapod_create", "hapod_push", "hapod_result", "hapod_node_stats", "hapod_profile", "hapod_last_error",
            "hapod_destroy", "hapod_trim_pool",
            "hapod_gram", "hapod_eig", "hapod_truncate", "hapod_modes", "hapod_pod", "hapod_gram_noalloc",
            "hapod_synth_snapshots", "hapod_result_right", "hapod_autotune", "hapod_autotune_clear")


def _stream(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(st: int, ctx=None, allow_warn: bool = True) -> int:
    if st == HAPOD_OK or (allow_warn and st >= HAPOD_WARN_NOCONVERGE):
        return st
    msg = _lib.hapod_last_error(ctx)
    raise HapodError(st, msg.decode() if msg else "")


def _colmajor(X: torch.Tensor) -> Tuple[int, int, int]:
    """(n, m, ld) of an n x m column-major view (stride(0) == 1)."""
    if X.dim() != 2 or X.stride(0) != 1 or not X.is_cuda:
        raise ValueError("expected a 2-D CUDA tensor in column-major layout (stride(0) == 1)")
    n, m = X.shape
    return n, m, max(X.stride(1), n)


def colmajor_empty(n: int, m: int, dtype, device) -> torch.Tensor:
    """n x m column-major CUDA tensor (storage is m x n row-major)."""
    return torch.empty((m, n), dtype=dtype, device=device).t()


# ------------------------------------------------------------------ context
class Context:
    """Owns one hapod_ctx.  ``parent``/``leaf_cols`` describe the rooted tree."""

    def __init__(self, parent: Sequence[int], leaf_cols: Sequence[int], eps: float, omega: float, n_rows: int,
                 precision: int = HAPOD_FP64, eps_override: Optional[Sequence[float]] = None,
                 max_pending_leaves: int = 0, stream: Optional[torch.cuda.Stream] = None, flags: int = 0):
        N = len(parent)
        self._parent = (ctypes.c_int32 * N)(*parent)
        self._cols = (ctypes.c_int64 * N)(*[int(c) for c in leaf_cols])
        has_child = [False] * N
        for p_ in parent:
            if p_ >= 0:
                has_child[p_] = True
        self._is_leaf = [not h for h in has_child]
        self._ovr = (ctypes.c_double * N)(*eps_override) if eps_override is not None else None
        tree = hapod_tree(N, self._parent, self._cols)
        tol = hapod_tol(float(eps), float(omega),
                        ctypes.cast(self._ovr, ctypes.POINTER(ctypes.c_double)) if self._ovr else None,
                        int(precision), int(max_pending_leaves), int(flags))
        self.precision = precision
        self.n = int(n_rows)
        self.stream = stream
        self.ctx = ctypes.c_void_p()
        _check(_lib.hapod_create(ctypes.byref(tree), ctypes.byref(tol), self.n, ctypes.c_void_p(_stream(stream)),
                                 ctypes.byref(self.ctx)), None)

    def close(self):
        if self.ctx:
            _lib.hapod_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hapod_create(parent, leaf_cols, eps, omega, n_rows, precision=HAPOD_FP64, eps_override=None,
                 max_pending_leaves=0, stream=None, flags=0) -> Context:
    return Context(parent, leaf_cols, eps, omega, n_rows, precision, eps_override, max_pending_leaves, stream, flags)


def hapod_push(ctx: Context, leaf: int, X: torch.Tensor) -> int:
    """Push the n x ncols column-major snapshots of ``leaf`` (device tensor)."""
    if X.dtype != DTYPE[ctx.precision]:
        raise TypeError(f"snapshots must be {DTYPE[ctx.precision]} for this precision")
    n, m, ld = _colmajor(X) if X.numel() else (ctx.n, X.shape[1], ctx.n)
    if n != ctx.n:
        raise ValueError("row count differs from n_rows")
    return _check(_lib.hapod_push(ctx.ctx, int(leaf), ctypes.c_void_p(X.data_ptr() if X.numel() else 0), ld, m),
                  ctx.ctx)


def hapod_result(ctx: Context, device=None):
    """Returns (sigma: float64 CPU tensor, modes: n x k column-major CUDA tensor, status)."""
    k = ctypes.c_int64(0)
    _check(_lib.hapod_result(ctx.ctx, ctypes.byref(k), None, None, 0), ctx.ctx)
    kk = k.value
    device = device or torch.device("cuda", torch.cuda.current_device())
    sigma = torch.zeros(max(kk, 0), dtype=torch.float64)
    modes = colmajor_empty(ctx.n, max(kk, 0), DTYPE[ctx.precision], device)
    sp = ctypes.cast(sigma.data_ptr(), ctypes.POINTER(ctypes.c_double)) if kk else None
    st = _check(_lib.hapod_result(ctx.ctx, ctypes.byref(k), sp, ctypes.c_void_p(modes.data_ptr() if kk else 0),
                                  ctx.n), ctx.ctx)
    return sigma, modes, st


def hapod_result_right(ctx: Context, k: int, device=None) -> torch.Tensor:
    """Right factor Lambda~ (|S| x k FP64, column-major CUDA tensor) of the low-rank
    approximation S ~ U diag(sigma) Lambda~^T (context created with
    HAPOD_FLAG_RIGHT_VECTORS, after hapod_result)."""
    S = int(sum(ctx._cols[a] for a in range(len(ctx._cols)) if ctx._is_leaf[a]))
    device = device or torch.device("cuda", torch.cuda.current_device())
    W = colmajor_empty(S, max(k, 0), torch.float64, device)
    _check(_lib.hapod_result_right(ctx.ctx, ctypes.c_void_p(W.data_ptr() if k > 0 else 0), S), ctx.ctx)
    return W


def hapod_node_stats(ctx: Context, node: int) -> dict:
    info = hapod_node_info()
    _check(_lib.hapod_node_stats(ctx.ctx, int(node), ctypes.byref(info)), ctx.ctx)
    return {f: getattr(info, f) for f, _ in hapod_node_info._fields_}


def hapod_profile(ctx: Context) -> dict:
    """Per-step device time (ms), launches and algorithmic bytes/flops (HAPOD_FLAG_PROFILE)."""
    info = hapod_profile_info()
    _check(_lib.hapod_profile(ctx.ctx, ctypes.byref(info)), ctx.ctx)
    return {name: {"ms": info.ms[i], "launches": info.launches[i], "bytes": info.bytes[i], "flops": info.flops[i]}
            for i, name in enumerate(PROFILE_STEPS)}


def hapod_last_error(ctx: Optional[Context] = None) -> str:
    r = _lib.hapod_last_error(ctx.ctx if ctx is not None else None)
    return r.decode() if r else ""


def hapod_destroy(ctx: Context) -> None:
    ctx.close()


def hapod_trim_pool(stream=None) -> None:
    """Return the device memory the library's pool keeps cached between contexts."""
    _check(_lib.hapod_trim_pool(ctypes.c_void_p(_stream(stream))))


# ------------------------------------------------------------------ single-node steps
def hapod_gram(X: torch.Tensor, precision: int = HAPOD_FP64, stream=None) -> torch.Tensor:
    n, m, ld = _colmajor(X)
    G = torch.empty((m, m), dtype=torch.float64, device=X.device)
    _check(_lib.hapod_gram(precision, n, m, ctypes.c_void_p(X.data_ptr()), ld, ctypes.c_void_p(G.data_ptr()),
                           ctypes.c_void_p(_stream(stream))))
    return G  # symmetric: row- or column-major alike


def hapod_gram_noalloc(X: torch.Tensor, G: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """FP64 Gram without device allocation inside the library (see include/hapod.h);
    pass a preallocated m x m float64 ``G`` to avoid the allocation here as well."""
    n, m, ld = _colmajor(X)
    if G is None:
        G = torch.empty((m, m), dtype=torch.float64, device=X.device)
    _check(_lib.hapod_gram_noalloc(n, m, ctypes.c_void_p(X.data_ptr()), ld, ctypes.c_void_p(G.data_ptr()),
                                   ctypes.c_void_p(_stream(stream))))
    return G


def hapod_eig(G: torch.Tensor, precision: int = HAPOD_FP64, stream=None):
    """Returns (lambda descending, V column-major m x m, sweeps, status)."""
    m = G.shape[0]
    Gc = G.contiguous()
    lam = torch.empty(m, dtype=torch.float64, device=G.device)
    V = colmajor_empty(m, m, torch.float64, G.device)
    sw = ctypes.c_int32(0)
    st = _check(_lib.hapod_eig(precision, m, ctypes.c_void_p(Gc.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                               ctypes.c_void_p(V.data_ptr()), ctypes.byref(sw), ctypes.c_void_p(_stream(stream))))
    return lam, V, sw.value, st


def hapod_truncate(lam: torch.Tensor, eps: float, stream=None) -> Tuple[int, float]:
    N = ctypes.c_int64(0)
    tail = ctypes.c_double(0.0)
    _check(_lib.hapod_truncate(lam.numel(), ctypes.c_void_p(lam.data_ptr()), float(eps), ctypes.byref(N),
                               ctypes.byref(tail), ctypes.c_void_p(_stream(stream))))
    return N.value, tail.value


def hapod_modes(X: torch.Tensor, V: torch.Tensor, N: int, scale: Optional[torch.Tensor] = None,
                precision: int = HAPOD_FP64, stream=None) -> torch.Tensor:
    n, m, ld = _colmajor(X)
    if V.stride(0) != 1 or V.dtype != torch.float64:
        raise ValueError("V must be a column-major float64 tensor")
    Y = colmajor_empty(n, N, X.dtype, X.device)
    _check(_lib.hapod_modes(precision, n, m, ctypes.c_void_p(X.data_ptr()), ld, ctypes.c_void_p(V.data_ptr()),
                            max(V.stride(1), m), N, ctypes.c_void_p(scale.data_ptr() if scale is not None else 0),
                            ctypes.c_void_p(Y.data_ptr() if N else 0), n, ctypes.c_void_p(_stream(stream))))
    return Y


def hapod_pod(X: torch.Tensor, eps: float, precision: int = HAPOD_FP64, stream=None):
    """POD(S, eps) of one node: returns (N, sigma[:N] (CUDA f64), Y n x N column-major, tail, status)."""
    n, m, ld = _colmajor(X)
    sigma = torch.zeros(max(m, 1), dtype=torch.float64, device=X.device)
    Y = colmajor_empty(n, max(m, 1), X.dtype, X.device)
    N = ctypes.c_int64(0)
    tail = ctypes.c_double(0.0)
    st = _check(_lib.hapod_pod(precision, n, m, ctypes.c_void_p(X.data_ptr()), ld, float(eps), ctypes.byref(N),
                               ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(Y.data_ptr()), n,
                               ctypes.byref(tail), ctypes.c_void_p(_stream(stream))))
    k = N.value
    return k, sigma[:k], Y[:, :k], tail.value, st


# ------------------------------------------------------------------ input generation
def synth_params(seed: int, harmonic_amp, nu: float, speed: float, pulse_centre=(), pulse_amp=(),
                 pulse_width: float = 0.01) -> hapod_synth_params:
    p = hapod_synth_params()
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.nu, p.speed = float(nu), float(speed)
    if len(harmonic_amp) != 32 or len(pulse_centre) != len(pulse_amp) or len(pulse_amp) > SYNTH_MAX_PULSES:
        raise ValueError("32 harmonic amplitudes and at most 64 pulses (centre, amplitude) expected")
    for k, a in enumerate(harmonic_amp):
        p.harmonic_amp[k] = float(a)
    p.num_pulses = len(pulse_amp)
    p.pulse_width = float(pulse_width)
    for q, (c, a) in enumerate(zip(pulse_centre, pulse_amp)):
        p.pulse_centre[q] = float(c)
        p.pulse_amp[q] = float(a)
    return p


def hapod_synth_snapshots(params: hapod_synth_params, n: int, col0: int, ncols: int, out: torch.Tensor,
                          t_out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Fill the n x ncols column-major CUDA tensor ``out`` (float32 or float64) with
    columns col0 .. col0 + ncols - 1 of the travelling-pulse trajectory."""
    nn, m, ld = _colmajor(out) if out.numel() else (n, ncols, n)
    if nn != n or m != ncols or out.dtype not in (torch.float32, torch.float64):
        raise ValueError("out must be an n x ncols float32/float64 column-major CUDA tensor")
    if t_out is not None and (t_out.dtype != torch.float64 or t_out.numel() < ncols or not t_out.is_cuda):
        raise ValueError("t_out must be a CUDA float64 tensor of ncols entries")
    _check(_lib.hapod_synth_snapshots(ctypes.byref(params), int(n), int(col0), int(ncols),
                                      0 if out.dtype == torch.float32 else 1,
                                      ctypes.c_void_p(out.data_ptr() if out.numel() else 0), ld,
                                      ctypes.c_void_p(t_out.data_ptr() if t_out is not None else 0),
                                      ctypes.c_void_p(_stream(stream))))
    return out


# ------------------------------------------------------------------ autotuner
def hapod_autotune(X: torch.Tensor, precision: int, stream=None):
    """Time the Gram of the n x m column-major node X at split factors 50/100/200/400 %
    and keep the fastest for its (form, m, n) bucket; returns (percent, [ms x 4])."""
    n, m, ld = _colmajor(X)
    pct = ctypes.c_int32(0)
    ms = (ctypes.c_double * 4)()
    _check(_lib.hapod_autotune(int(precision), n, m, ctypes.c_void_p(X.data_ptr()), ld, ctypes.byref(pct), ms,
                               ctypes.c_void_p(_stream(stream))))
    return pct.value, list(ms)


def hapod_autotune_clear() -> None:
    _lib.hapod_autotune_clear()


def eps_star_to_global(eps_star: float, num_snapshots: int) -> float:
    """Global l2 tolerance eps = sqrt(|S|) eps* (Thm. cor:hapod_bound's mean error)."""
    return math.sqrt(num_snapshots) * eps_star
