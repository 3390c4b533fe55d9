"""Bounded device-side waits: with the debug-only budget HAPOD_DEBUG_WAIT_CYCLES=1 the
first mbarrier wait of each tensor-core kernel that is not already satisfied runs
out on a healthy kernel.  The call must return HAPOD_ERR_TIMEOUT (no hang, no fault),
and the next call in the same process, with the budget back to normal, must succeed
with correct results -- which it can only do if the timed-out CTAs drained their
copies and MMAs and freed their tensor memory.

Runs in a child process so that the environment variable and any state it leaves
stay out of the other tests.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os
    import torch
    from paper_1607_05210_gb300 import hapod as H

    torch.manual_seed(5)
    n, m = 1 << 16, 96
    X32 = torch.randn((m, n), dtype=torch.float32, device="cuda").t()   # n x m column-major
    X64 = torch.randn((m, n), dtype=torch.float64, device="cuda").t()
    V = torch.randn((12, m), dtype=torch.float64, device="cuda").t() / 8
    calls = {
        "gram_bf16x3": lambda: H.hapod_gram(X32, H.HAPOD_MIXED_BF16X3),
        "gram_tf32x3": lambda: H.hapod_gram(X32, H.HAPOD_MIXED_TF32X3),
        "gram_fixed3": lambda: H.hapod_gram(X32, H.HAPOD_MIXED_FX3),
        "gram_digit_slice": lambda: H.hapod_gram(X64, H.HAPOD_FP64_OZAKI),
        "modes_digit_slice": lambda: H.hapod_modes(X64, V, 12, None, H.HAPOD_FP64_OZAKI),
    }
    os.environ["HAPOD_DEBUG_WAIT_CYCLES"] = "1"
    for name, f in calls.items():
        try:
            f()
            torch.cuda.synchronize()
            print("NO_TIMEOUT", name, flush=True)
        except H.HapodError as e:
            assert e.status == H.HAPOD_ERR_TIMEOUT, (name, e.status)
            print("TIMEOUT", name, flush=True)
    del os.environ["HAPOD_DEBUG_WAIT_CYCLES"]
    G_ref = (X32.double().t() @ X32.double())
    d = torch.sqrt(torch.diag(G_ref))
    for name in ("gram_bf16x3", "gram_tf32x3", "gram_fixed3"):
        G = calls[name]()
        err = float(torch.max(torch.abs(G - G_ref) / torch.outer(d, d)))
        assert err <= 1e-5, (name, err)
    G = calls["gram_digit_slice"]()
    G_ref = X64.t() @ X64
    d = torch.sqrt(torch.diag(G_ref))
    assert float(torch.max(torch.abs(G - G_ref) / torch.outer(d, d))) <= 1e-12
    Y = calls["modes_digit_slice"]()
    Y_ref = X64 @ V
    assert float(torch.max(torch.abs(Y - Y_ref))) <= 1e-10 * float(torch.max(torch.abs(Y_ref)))
    torch.cuda.synchronize()
    print("RECOVERED", flush=True)
""")


def test_bounded_wait_times_out_and_the_context_recovers(cuda_ok):
    env = dict(os.environ)
    env.pop("HAPOD_DEBUG_WAIT_CYCLES", None)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    print(r.stdout)
    print(r.stderr[-3000:])
    assert r.returncode == 0
    for name in ("gram_bf16x3", "gram_tf32x3", "gram_fixed3", "gram_digit_slice", "modes_digit_slice"):
        assert f"TIMEOUT {name}" in r.stdout
    assert "RECOVERED" in r.stdout
