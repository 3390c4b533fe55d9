"""Host pins of the seeded input generators (no GPU): the Philox4x32-10 twin against
the published known-answer vectors, the snapshot-time mapping, and the travelling-
pulse snapshots against their defining formula evaluated term by term."""
import math
import os

import numpy as np

from paper_1607_05210_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = synth.philox4x32_10([[w[0]], [w[1]], [w[2]], [w[3]]], (w[4], w[5]))
        assert [int(v) for v in out[:, 0]] == w[6:10]


def test_philox_times_are_per_column_and_uniform():
    t = synth.philox_times(1607, 0, 4096)
    assert np.all((t >= 0.0) & (t < 1.0))
    # any column range reproduces the same times (stream chunks)
    assert np.array_equal(synth.philox_times(1607, 1000, 96), t[1000:1096])
    # counters above 2^32 use the high word
    hi = synth.philox_times(1607, (1 << 32) + 5, 2)
    assert not np.array_equal(hi, t[5:7])
    # 53-bit uniforms: mean and variance of U[0, 1) within 5 standard errors
    assert abs(t.mean() - 0.5) < 5 * math.sqrt(1 / 12 / t.size)
    assert abs(t.var() - 1 / 12) < 5 * 0.0745 / math.sqrt(t.size)
    # the mapping of the first two output words
    z = np.zeros(1, dtype=np.uint64)
    w = synth.philox4x32_10([z + 7, z, z, z], (1607, 0))
    assert t[7] == ((int(w[0, 0]) << 21) | (int(w[1, 0]) >> 11)) * 2.0 ** -53


def _by_definition(n, col0, ncols, P):
    t = synth.philox_times(P["seed"], col0, ncols)
    x = 2.0 * math.pi * np.arange(n) / n
    k = np.arange(1, 33)
    X = np.zeros((n, ncols))
    for j in range(ncols):
        X[:, j] = np.sum(P["harmonic_amp"] * np.exp(-P["nu"] * k * k * t[j]) *
                         np.sin(k * (x[:, None] - P["speed"] * t[j])), axis=1)
        for c, a in zip(P["pulse_centre"], P["pulse_amp"]):
            d = np.abs(x - np.mod(c + P["speed"] * t[j], 2.0 * math.pi))
            d = np.minimum(d, 2.0 * math.pi - d)
            X[:, j] += a * np.exp(-d * d / (2.0 * P["pulse_width"] ** 2))
    return X


def test_pulse_snapshots_follow_their_definition():
    P = synth.pulse_workload(11)
    assert len(P["pulse_amp"]) == 64 and np.allclose(P["pulse_amp"] * np.arange(1, 65), 1.0)
    for n, col0, ncols in [(4096, 0, 8), (1000, 77, 5), (5, 3, 4)]:
        X = synth.pulse_snapshots(n, col0, ncols, P, np.float64)
        ref = _by_definition(n, col0, ncols, P)
        # terms beyond 9 w are left out: each is below exp(-40.5) of its amplitude
        assert np.max(np.abs(X - ref)) <= 64 * math.exp(-40.5) + 1e-13


def test_pulse_wraps_around_the_period():
    P = synth.pulse_workload(3, num_pulses=1)
    P["harmonic_amp"] = np.zeros(32)
    P["pulse_centre"] = np.array([2.0 * math.pi - 1e-3])
    P["speed"] = 0.0  # the pulse sits at 2 pi - 1e-3 for every t
    n = 1 << 14
    X = synth.pulse_snapshots(n, 0, 2, P, np.float64)
    x = 2.0 * math.pi * np.arange(n) / n
    d = np.minimum(np.abs(x - P["pulse_centre"][0]), 2.0 * math.pi - np.abs(x - P["pulse_centre"][0]))
    assert np.allclose(X[:, 0], np.where(d <= 0.09, np.exp(-d * d / 2e-4), 0.0), rtol=0, atol=1e-15)
    assert X[0, 0] > 0.99 and X[n // 2, 0] == 0.0  # the part past 2 pi shows up at x = 0
