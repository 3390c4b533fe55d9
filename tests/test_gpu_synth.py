"""The library's device snapshot generator (hapod_synth_snapshots) against its host
twin in synth.py: snapshot times bit for bit (Philox4x32-10 is integer arithmetic),
the field within the FP32 evaluation error, column ranges reproducible on their own,
and the FP64 output holding exactly the FP32 values.

Field tolerance: the device sums 64 Fourier terms in FP32 from FP32-rounded
coefficients and sincospif values (each within 2^-23 relative), and each pulse term
from an FP32 distance and expf: |X_dev - X_host| <= 2^-17 (sum_k |a_k| + sum_p A_p)
covers 64 accumulated roundings of 2^-24 with margin."""
import math

import numpy as np
import pytest
import torch

from paper_1607_05210_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H(cuda_ok):
    from paper_1607_05210_gb300 import hapod

    return hapod


def _gen(H, P, n, col0, ncols, dtype=torch.float32, ld=None):
    ld = ld or n
    buf = torch.full((ncols, ld), float("nan"), dtype=dtype, device="cuda")
    t = torch.empty(ncols, dtype=torch.float64, device="cuda")
    H.hapod_synth_snapshots(H.synth_params(**P), n, col0, ncols, buf[:, :n].t(), t_out=t)
    torch.cuda.synchronize()
    return buf, t


@pytest.mark.parametrize("n,col0,ncols,ld", [(4096, 0, 64, 4096), (1000, 77, 33, 1003), (1 << 16, 1 << 20, 40, 1 << 16),
                                             (257, 5, 1, 260), (3, 0, 7, 3), (1 << 20, 0, 3, 1 << 20)])
def test_device_generator_matches_host_twin(H, n, col0, ncols, ld):
    P = synth.pulse_workload(1607 + n)
    buf, t = _gen(H, P, n, col0, ncols, ld=ld)
    assert np.array_equal(t.cpu().numpy(), synth.philox_times(P["seed"], col0, ncols))
    X = buf[:, :n].t().double().cpu().numpy()
    ref = synth.pulse_snapshots(n, col0, ncols, P, np.float64)
    scale = float(np.sum(np.abs(P["harmonic_amp"])) + np.sum(P["pulse_amp"]))
    err = np.max(np.abs(X - ref))
    print(f"n={n} col0={col0} ncols={ncols}: max err {err:.3e} (scale {scale:.2f})")
    assert err <= 2.0 ** -17 * scale
    if ld > n:  # padding rows untouched
        assert torch.isnan(buf[:, n:]).all()


def test_column_ranges_and_precisions_agree_bit_for_bit(H):
    P = synth.pulse_workload(3)
    n = 50_000
    full, _ = _gen(H, P, n, 0, 96)
    part, _ = _gen(H, P, n, 40, 24)
    assert torch.equal(full[40:64], part)
    d, _ = _gen(H, P, n, 0, 96, dtype=torch.float64)
    assert torch.equal(d, full.double())


def test_pulses_only_and_the_periodic_wrap(H):
    P = synth.pulse_workload(5, num_pulses=3)
    P["harmonic_amp"] = np.zeros(32)
    P["pulse_centre"] = np.array([2.0 * math.pi - 1e-3, 0.5, 3.0])
    n = 1 << 15
    buf, _ = _gen(H, P, n, 0, 16)
    X = buf.t().double().cpu().numpy()
    ref = synth.pulse_snapshots(n, 0, 16, P, np.float64)
    assert np.max(np.abs(X - ref)) <= 2.0 ** -20 * np.sum(P["pulse_amp"])
    # the same 9 w windows, up to entries at the cut itself (below exp(-40.4) A_p)
    differ = (X != 0) != (ref != 0)
    assert np.all(np.maximum(np.abs(X), np.abs(ref))[differ] <= math.exp(-40.4))
    assert np.count_nonzero(differ) <= 4


def test_invalid_arguments(H):
    P = H.synth_params(**synth.pulse_workload(1))
    lib = H._lib
    X = torch.empty((4, 100), device="cuda")
    assert lib.hapod_synth_snapshots(None, 100, 0, 4, 0, X.data_ptr(), 100, None, None) == H.HAPOD_ERR_INVALID
    import ctypes

    for n, col0, ncols, dt, ld in [(0, 0, 4, 0, 100), (100, -1, 4, 0, 100), (100, 0, 4, 2, 100), (100, 0, 4, 0, 99)]:
        assert lib.hapod_synth_snapshots(ctypes.byref(P), n, col0, ncols, dt, X.data_ptr(), ld, None,
                                         None) == H.HAPOD_ERR_INVALID
    P.num_pulses = 65
    assert lib.hapod_synth_snapshots(ctypes.byref(P), 100, 0, 4, 0, X.data_ptr(), 100, None,
                                     None) == H.HAPOD_ERR_INVALID
    P.num_pulses = 0
    assert lib.hapod_synth_snapshots(ctypes.byref(P), 100, 0, 0, 0, None, 100, None, None) == H.HAPOD_OK
