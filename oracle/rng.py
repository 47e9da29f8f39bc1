"""Counter-based parameter stream (oracle side).

The paper draws the fixed hidden-layer parameters from U(-a, a) (§4.1 "Neural
network architecture and weight initialisation") with JAX's generator, which is
not reproducible from the text.  Both sides of this project therefore use
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; constants as in Vigna's public-domain reference
``splitmix64.c``), each side implementing it from that published definition.

Stream definition (the contract both sides follow):

* output i (i >= 0) of the generator seeded with ``seed`` is
  ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64)``;
* column q (global feature index, §3 "Indexing conventions", 0-based) of a
  problem in ``dim`` dimensions owns outputs ``i = q * (dim + 1) + p`` with
  p = 0..dim-1 the input weights and p = dim the bias;
* a 24-bit uniform u = (z >> 40) * 2^-24 in [0, 1) maps to a * (2u - 1).

Pinned by the published SplitMix64 output sequences (tests/test_oracle_rng.py).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (two xor-shift-multiply rounds and a final xor-shift)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_at(seed: int, index) -> np.ndarray:
    """Output number ``index`` (0-based) of SplitMix64 seeded with ``seed``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GOLDEN
    return splitmix64_mix(state)


def uniform24(seed: int, index) -> np.ndarray:
    """24-bit uniform in [0, 1) from output ``index``."""
    z = splitmix64_at(seed, index)
    return (z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def draw_parameters(seed: int, n_columns: int, dim: int, a: float):
    """Fixed random parameters of every column: W (n_columns, dim), b (n_columns,).

    Both ~ U(-a, a) (§4.1).  With a = 1 every value is exactly representable
    in float32 (24-bit uniforms), so float32 and float64 paths see the same
    parameters.
    """
    q = np.arange(n_columns, dtype=np.uint64)[:, None]
    p = np.arange(dim + 1, dtype=np.uint64)[None, :]
    u = uniform24(seed, q * np.uint64(dim + 1) + p)
    v = a * (2.0 * u - 1.0)
    return v[:, :dim].copy(), v[:, dim].copy()
