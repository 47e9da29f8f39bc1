"""Pins of the oracle's windows (Eq. window_func) and decomposition (§4.1)."""
import math

import numpy as np
import pytest

from oracle import decomposition as D
from oracle import windows as Wn


CASES = [
    (1, (16,), 2.0, "cell"),
    (1, (1, 2, 4, 8), 2.0, "cell"),
    (1, (20,), 2.9, "endpoint"),
    (2, (1, 2, 4), 2.0, "cell"),
    (2, (3, 5), 2.9, "cell"),
]


def _levels(dim, levels, delta, placement, K=4):
    lo = (0.0,) * dim
    hi = (1.0,) * dim
    return D.build_levels(dim, lo, hi, levels, delta, K, placement)


@pytest.mark.parametrize("dim,levels,delta,placement", CASES)
def test_partition_of_unity_and_vanishing_derivatives(dim, levels, delta, placement):
    rng = np.random.default_rng(0)
    X = rng.random((400, dim))
    for lev in _levels(dim, levels, delta, placement):
        w = Wn.level_windows(X, lev, dim)
        assert np.allclose(w["om"].sum(axis=1), 1.0, atol=1e-14)
        scale_d = max(math.pi / s for s in lev.sigma)
        assert np.allclose(w["dom"].sum(axis=1), 0.0, atol=1e-12 * scale_d)
        assert np.allclose(w["ddom"].sum(axis=1), 0.0, atol=1e-11 * scale_d ** 2)


def test_window_peak_value_is_four_to_the_d():
    for dim in (1, 2):
        lev = _levels(dim, (4,), 2.0, "cell")[0]
        # the centre of subdomain j=5 (2-D) or j=1 (1-D)
        j = 5 if dim == 2 else 1
        ji = D.subdomain_multi_index(lev, dim, j)
        mu = np.array([[lev.mu[i][ji[i]] for i in range(dim)]])
        w = Wn.level_windows(mu, lev, dim)
        assert w["what"][0, j] == pytest.approx(4.0 ** dim, rel=1e-15)


def test_factor_derivatives_complex_step_and_fd():
    mu, sigma = 0.3, 0.17
    x = np.linspace(mu - 0.95 * sigma, mu + 0.95 * sigma, 41)
    f, df, ddf = Wn.window_factor_1d(x, mu, sigma)
    h = 1e-30
    fc, dfc, _ = Wn.window_factor_1d(x + 1j * h, mu, sigma)
    assert np.allclose(fc.imag / h, df, rtol=1e-12, atol=1e-10)
    assert np.allclose(dfc.imag / h, ddf, rtol=1e-12, atol=1e-8)
    e = 1e-6
    fp, _, _ = Wn.window_factor_1d(x + e, mu, sigma)
    fm, _, _ = Wn.window_factor_1d(x - e, mu, sigma)
    assert np.allclose((fp - fm) / (2 * e), df, rtol=1e-7, atol=1e-6)
    # on the edge of the open support and outside it everything vanishes
    mu2, sigma2 = 0.25, 0.125          # dyadic, so mu +- sigma is exact
    out = np.array([mu2 - sigma2, mu2 + sigma2, mu2 + 1.5 * sigma2])
    for arr in Wn.window_factor_1d(out, mu2, sigma2):
        assert np.all(arr == 0.0)


@pytest.mark.parametrize("dim,levels,delta,placement", CASES)
def test_normalised_window_derivatives_complex_step(dim, levels, delta, placement):
    """Quotient-rule derivatives of w_j = w_hat_j / S against the complex step."""
    rng = np.random.default_rng(1)
    X = 0.05 + 0.9 * rng.random((60, dim))
    h = 1e-30
    for lev in _levels(dim, levels, delta, placement):
        w = Wn.level_windows(X, lev, dim)
        for i in range(dim):
            Xc = X.astype(complex)
            Xc[:, i] += 1j * h
            wc = Wn.level_windows(Xc, lev, dim)
            scale = math.pi / lev.sigma[i]
            assert np.allclose(wc["om"].imag / h, w["dom"][:, :, i], rtol=1e-10, atol=1e-11 * scale)
            assert np.allclose(wc["dom"][:, :, i].imag / h, w["ddom"][:, :, i],
                               rtol=1e-9, atol=1e-10 * scale ** 2)


def test_support_mask_open_and_consistent_with_values():
    dim = 2
    lev = _levels(dim, (1, 2, 4), 2.0, "cell")[2]
    rng = np.random.default_rng(2)
    X = rng.random((2000, dim))
    m = Wn.support_mask(X, lev, dim)
    w = Wn.level_windows(X, lev, dim)
    assert np.array_equal(m, w["what"] > 0)
    # with delta = 2 and cell-centred subdomains each coordinate is covered by 1 or 2 subdomains
    assert set(np.unique(m.sum(axis=1))) <= {1, 2, 4}


def test_column_offsets_follow_indexing_convention():
    levels = _levels(2, (1, 2, 4), 2.0, "cell", K=8)
    assert [l.col_offset for l in levels] == [0, 8, 8 + 4 * 8]
    assert [l.n_sub for l in levels] == [1, 4, 16]
    lev = levels[2]
    assert D.subdomain_multi_index(lev, 2, 6) == (2, 1)  # j = j_y * n + j_x
    assert [j for j, _ in D.all_subdomains(lev, 2)] == list(range(16))
    assert [ji for _, ji in D.all_subdomains(lev, 2)][6] == (2, 1)


def test_geometry_closed_form():
    lev = _levels(1, (16,), 2.0, "cell")[0]
    assert np.allclose(lev.mu[0], (np.arange(16) + 0.5) / 16)
    assert lev.sigma[0] == pytest.approx(1 / 16)
    lev = _levels(1, (20,), 2.9, "endpoint")[0]
    assert np.allclose(lev.mu[0], np.arange(20) / 19)
    assert lev.sigma[0] == pytest.approx(2.9 / 19 / 2)
