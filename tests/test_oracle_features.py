"""Pins of the oracle's tanh random features (§3, h = 1) and derivatives."""
import math

import numpy as np

from oracle import features as F


def test_feature_values_are_tanh_of_affine_normalised_input():
    rng = np.random.default_rng(0)
    Z = rng.uniform(-1, 1, (7, 2))
    W = rng.uniform(-1, 1, (5, 2))
    b = rng.uniform(-1, 1, 5)
    phi, _, _, s = F.features(Z, W, b, np.array([0.1, 0.2]))
    for n in range(7):
        for k in range(5):
            ref = math.tanh(W[k, 0] * Z[n, 0] + W[k, 1] * Z[n, 1] + b[k])
            assert abs(phi[n, k] - ref) <= 1e-16 + 1e-15 * abs(ref)


def test_feature_derivatives_complex_step():
    """d/dx of x -> tanh(w.(x - mu)/sigma + b) by complex step, 2nd derivative by complex step of the 1st."""
    rng = np.random.default_rng(1)
    mu = np.array([0.4, 0.6])
    sig = np.array([0.125, 0.25])
    X = mu + rng.uniform(-1, 1, (30, 2)) * sig
    W = rng.uniform(-1, 1, (6, 2))
    b = rng.uniform(-1, 1, 6)
    phi, dphi, ddphi, _ = F.features((X - mu) / sig, W, b, sig)
    h = 1e-30
    for i in range(2):
        Xc = X.astype(complex)
        Xc[:, i] += 1j * h
        phic, dphic, _, _ = F.features((Xc - mu) / sig, W, b, sig)
        assert np.allclose(phic.imag / h, dphi[:, :, i], rtol=1e-12, atol=1e-13)
        assert np.allclose(dphic[:, :, i].imag / h, ddphi[:, :, i], rtol=1e-11, atol=1e-11)


def test_feature_second_derivative_central_difference():
    mu = np.array([0.5])
    sig = np.array([0.0625])
    W = np.array([[0.9], [-0.3]])
    b = np.array([0.2, -0.7])
    x = np.linspace(0.45, 0.55, 11)[:, None]
    e = 1e-5
    phi, dphi, ddphi, _ = F.features((x - mu) / sig, W, b, sig)
    pp = F.features((x + e - mu) / sig, W, b, sig)[0]
    pm = F.features((x - e - mu) / sig, W, b, sig)[0]
    assert np.allclose((pp - 2 * phi + pm) / e ** 2, ddphi[:, :, 0], rtol=1e-4, atol=1e-3)
