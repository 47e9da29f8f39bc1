"""Pins of the oracle's SplitMix64 parameter stream against published outputs."""
import os

import numpy as np

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        vals = [int(v) for v in line.split()]
        rows.append((vals[0], vals[1:]))
    return rows


def test_splitmix64_published_sequences():
    for seed, outs in _golden():
        got = rng.splitmix64_at(seed, np.arange(len(outs)))
        assert [int(v) for v in got] == outs


def test_counter_access_matches_sequential_state():
    # output i equals the i-th step of the sequential generator
    seed = 987654321
    state = seed
    M = (1 << 64) - 1
    for i in range(20):
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        assert int(rng.splitmix64_at(seed, i)) == z


def test_parameters_range_layout_and_float32_exact():
    W, b = rng.draw_parameters(seed=3, n_columns=4000, dim=2, a=1.0)
    assert W.shape == (4000, 2) and b.shape == (4000,)
    assert np.all(np.abs(W) <= 1.0) and np.all(np.abs(b) <= 1.0)
    # 24-bit uniforms: a = 1 values are exact in float32
    assert np.array_equal(W.astype(np.float32).astype(np.float64), W)
    assert np.array_equal(b.astype(np.float32).astype(np.float64), b)
    # layout: column q uses outputs q*(d+1) + p
    u = rng.uniform24(3, np.array([5 * 3 + 0, 5 * 3 + 1, 5 * 3 + 2]))
    assert np.allclose([W[5, 0], W[5, 1], b[5]], 2 * u - 1, rtol=0, atol=0)
    # roughly uniform: mean ~ 0, variance ~ 1/3
    allv = np.concatenate([W.ravel(), b])
    assert abs(allv.mean()) < 0.03
    assert abs(allv.var() - 1.0 / 3.0) < 0.02
