"""The C-ABI library loads and exports every symbol include/hapod.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hapod.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hapod_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1607_05210_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("hapod_create", "hapod_push", "hapod_result", "hapod_destroy", "hapod_node_stats", "hapod_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    from paper_1607_05210_gb300 import hapod as H

    assert set(H.EXPORTED) <= set(_declared())
    for n in H.EXPORTED:
        assert callable(getattr(H, n))


def test_invalid_arguments_are_rejected_without_a_gpu(lib_path):
    """Argument validation happens on the host before any CUDA call."""
    from paper_1607_05210_gb300 import hapod as H

    lib = H._lib
    out = ctypes.c_void_p()
    assert lib.hapod_create(None, None, 10, None, ctypes.byref(out)) == H.HAPOD_ERR_INVALID
    assert "null" in H.hapod_last_error()
    # two roots -> not a rooted tree
    par = (ctypes.c_int32 * 3)(-1, -1, 0)
    cols = (ctypes.c_int64 * 3)(5, 5, 5)
    tree = H.hapod_tree(3, par, cols)
    tol = H.hapod_tol(1e-3, 0.5, None, 0, 0, 0)
    assert lib.hapod_create(ctypes.byref(tree), ctypes.byref(tol), 10, None, ctypes.byref(out)) == H.HAPOD_ERR_TREE
    # a cycle 1 -> 2 -> 1 not connected to the root
    par = (ctypes.c_int32 * 3)(-1, 2, 1)
    tree = H.hapod_tree(3, par, cols)
    assert lib.hapod_create(ctypes.byref(tree), ctypes.byref(tol), 10, None, ctypes.byref(out)) == H.HAPOD_ERR_TREE
    # omega outside [0, 1]
    par = (ctypes.c_int32 * 3)(-1, 0, 0)
    tree = H.hapod_tree(3, par, cols)
    bad = H.hapod_tol(1e-3, 1.5, None, 0, 0, 0)
    assert lib.hapod_create(ctypes.byref(tree), ctypes.byref(bad), 10, None, ctypes.byref(out)) == H.HAPOD_ERR_INVALID
    assert out.value is None
    # step entry points
    assert lib.hapod_gram(7, 10, 3, None, 10, None, None) == H.HAPOD_ERR_INVALID
    assert lib.hapod_truncate(4, None, -1.0, None, None, None) == H.HAPOD_ERR_INVALID


def test_trim_pool_reports_a_missing_device(lib_path):
    """hapod_trim_pool returns a status, never aborts: without a usable CUDA device it
    is HAPOD_ERR_CUDA with the runtime's message in hapod_last_error()."""
    import torch

    from paper_1607_05210_gb300 import hapod as H

    st = H._lib.hapod_trim_pool(None)
    if torch.cuda.is_available():
        assert st == H.HAPOD_OK
    else:
        assert st == H.HAPOD_ERR_CUDA
        assert H.hapod_last_error()


def test_single_node_steps_validate_arguments_on_the_host(lib_path):
    """Each single-node entry point rejects bad arguments with HAPOD_ERR_INVALID and a
    message before touching CUDA (so the same status comes back with or without a GPU)."""
    from paper_1607_05210_gb300 import hapod as H

    lib = H._lib
    buf = (ctypes.c_double * 16)()
    N, tail = ctypes.c_int64(0), ctypes.c_double(0.0)
    calls = {
        "modes N > m": lambda: lib.hapod_modes(0, 10, 3, buf, 10, buf, 3, 5, None, buf, 10, None),
        "modes ldx < n": lambda: lib.hapod_modes(0, 10, 3, buf, 5, buf, 3, 2, None, buf, 10, None),
        "modes null X": lambda: lib.hapod_modes(0, 10, 3, None, 10, buf, 3, 2, None, buf, 10, None),
        "modes precision": lambda: lib.hapod_modes(9, 10, 3, buf, 10, buf, 3, 2, None, buf, 10, None),
        "eig null G": lambda: lib.hapod_eig(0, 3, None, buf, buf, None, None),
        "eig m > 13000": lambda: lib.hapod_eig(0, 13001, buf, buf, buf, None, None),
        "pod eps < 0": lambda: lib.hapod_pod(0, 10, 3, buf, 10, -1.0, ctypes.byref(N), buf, buf, 10,
                                             ctypes.byref(tail), None),
        "pod ldy < n": lambda: lib.hapod_pod(0, 10, 3, buf, 10, 1.0, ctypes.byref(N), buf, buf, 5,
                                             ctypes.byref(tail), None),
        "pod m > 13000": lambda: lib.hapod_pod(0, 20000, 13001, buf, 20000, 1.0, ctypes.byref(N), buf, buf, 20000,
                                               ctypes.byref(tail), None),
        "gram ldx < n": lambda: lib.hapod_gram(0, 10, 3, buf, 5, buf, None),
        "gram null G": lambda: lib.hapod_gram(0, 10, 3, buf, 10, None, None),
        "noalloc m > 2816": lambda: lib.hapod_gram_noalloc(10, 2817, buf, 10, buf, None),
        "truncate m < 0": lambda: lib.hapod_truncate(-1, buf, 1.0, ctypes.byref(N), ctypes.byref(tail), None),
    }
    for name, call in calls.items():
        assert call() == H.HAPOD_ERR_INVALID, name
        assert H.hapod_last_error(), name


def test_null_context_calls_fail_with_a_message(lib_path):
    from paper_1607_05210_gb300 import hapod as H

    lib = H._lib
    info = H.hapod_node_info()
    k = ctypes.c_int64(0)
    checks = [
        (lambda: lib.hapod_push(None, 0, None, 0, 0), "hapod_push"),
        (lambda: lib.hapod_result(None, ctypes.byref(k), None, None, 0), "hapod_result"),
        (lambda: lib.hapod_node_stats(None, 0, ctypes.byref(info)), "hapod_node_stats"),
    ]
    for call, name in checks:
        assert call() == H.HAPOD_ERR_INVALID
        assert name in H.hapod_last_error()
    lib.hapod_destroy(None)  # a no-op
