"""Partition-of-unity windows (oracle side).

§4.1 Eq. ``window_func``: the unnormalised window of subdomain j at level l is

    w_hat_j(x) = prod_i [1 + cos(pi (x_i - mu_ji) / sigma_ji)]^2

inside its support and zero outside (§3: windows vanish outside their
prescribed support), and the normalised window is w_j = w_hat_j / S with
S = sum_j w_hat_j over the subdomains of the same level, so that sum_j w_j = 1
(§3 "Problem and model definition").

Derivatives are written out from these definitions (chain rule for the 1-D
factor, product rule across dimensions, quotient rule for the normalisation).
The support is open: |theta| < pi (reading; the factor and its first three
theta-derivatives vanish at theta = +-pi, so only the sparsity pattern depends
on it).

Pinned by: partition of unity and its vanishing derivatives, w_hat(mu) = 4^d,
central finite differences and complex-step derivatives
(tests/test_oracle_windows.py).
"""
from __future__ import annotations

import math

import numpy as np


def window_factor_1d(x, mu, sigma):
    """1-D factor [1 + cos theta]^2 and its first two x-derivatives.

    theta = pi (x - mu) / sigma; zero (with derivatives) where |theta| >= pi.
    Returns (f, df, ddf), each broadcast over x and mu.
    """
    dx = np.asarray(x) - np.asarray(mu)
    theta = math.pi * dx / sigma
    inside = np.abs(dx) < sigma               # open support, |theta| < pi
    c = np.cos(theta)
    s = np.sin(theta)
    g = math.pi / sigma                       # d theta / dx
    f = (1.0 + c) ** 2
    df = -2.0 * (1.0 + c) * s * g
    ddf = (2.0 * s * s - 2.0 * (1.0 + c) * c) * g * g
    z = np.zeros_like(f)
    return np.where(inside, f, z), np.where(inside, df, z), np.where(inside, ddf, z)


def window_factor_1d_abs(x, mu, sigma):
    """Magnitudes of the terms of ``window_factor_1d`` (for error bounds)."""
    dx = np.asarray(x) - np.asarray(mu)
    theta = math.pi * dx / sigma
    inside = np.abs(dx) < sigma
    c = np.cos(theta)
    s = np.sin(theta)
    g = math.pi / sigma
    f = (1.0 + c) ** 2
    df = 2.0 * (1.0 + c) * np.abs(s) * g
    ddf = (2.0 * s * s + 2.0 * (1.0 + c) * np.abs(c)) * g * g
    z = np.zeros_like(f)
    return np.where(inside, f, z), np.where(inside, df, z), np.where(inside, ddf, z)


def level_windows(X, level, dim, with_abs=False):
    """Normalised windows of every subdomain of one level at points X.

    X: (n, dim).  Returns a dict with arrays of shape (n, J_l) (and (n, J_l, dim)
    for derivatives):
      'what'        w_hat_j                       (Eq. window_func numerator)
      'om'          w_j = w_hat_j / S
      'dom'[..., i] d_i w_j
      'ddom'[..., i] d_ii w_j
    and, with ``with_abs``, the magnitude sums 'dom_abs', 'ddom_abs' of the
    quotient-rule terms (used only to derive rounding tolerances).
    """
    n_pts = X.shape[0]
    n = level.n
    # per-dimension factors for every subdomain index along that dimension
    fac, dfac, ddfac = [], [], []
    fabs, dfabs, ddfabs = [], [], []
    for i in range(dim):
        f, df, ddf = window_factor_1d(X[:, i:i + 1], level.mu[i][None, :], level.sigma[i])
        fac.append(f); dfac.append(df); ddfac.append(ddf)
        if with_abs:
            fa, dfa, ddfa = window_factor_1d_abs(X[:, i:i + 1], level.mu[i][None, :], level.sigma[i])
            fabs.append(fa); dfabs.append(dfa); ddfabs.append(ddfa)

    J = n ** dim
    dt = np.result_type(np.asarray(X).dtype, np.float64)   # complex inputs allowed (complex step)
    what = np.ones((n_pts, J), dtype=dt)
    dwhat = np.ones((n_pts, J, dim), dtype=dt)
    ddwhat = np.ones((n_pts, J, dim), dtype=dt)
    dwhat_a = np.ones((n_pts, J, dim))
    ddwhat_a = np.ones((n_pts, J, dim))
    # subdomain j = sum_i j_i n^i ; product over dimensions (product rule)
    for i in range(dim):
        idx = (np.arange(J) // (n ** i)) % n
        what *= fac[i][:, idx]
        for k in range(dim):
            if k == i:
                dwhat[:, :, k] *= dfac[i][:, idx]
                ddwhat[:, :, k] *= ddfac[i][:, idx]
                if with_abs:
                    dwhat_a[:, :, k] *= dfabs[i][:, idx]
                    ddwhat_a[:, :, k] *= ddfabs[i][:, idx]
            else:
                dwhat[:, :, k] *= fac[i][:, idx]
                ddwhat[:, :, k] *= fac[i][:, idx]
                if with_abs:
                    dwhat_a[:, :, k] *= fabs[i][:, idx]
                    ddwhat_a[:, :, k] *= fabs[i][:, idx]

    # discarded subdomains (holes, §4.1) take no part in the level's windows
    if getattr(level, "keep", None) is not None:
        what = what * level.keep[None, :]
        dwhat = dwhat * level.keep[None, :, None]
        ddwhat = ddwhat * level.keep[None, :, None]
        dwhat_a = dwhat_a * level.keep[None, :, None]
        ddwhat_a = ddwhat_a * level.keep[None, :, None]
    # level sums (the normalisation of Eq. window_func)
    S = what.sum(axis=1)
    dS = dwhat.sum(axis=1)                  # (n, dim)
    ddS = ddwhat.sum(axis=1)
    Sx = S[:, None]
    om = what / Sx
    dom = dwhat / S[:, None, None] - what[:, :, None] * dS[:, None, :] / (S ** 2)[:, None, None]
    ddom = (ddwhat / S[:, None, None]
            - 2.0 * dwhat * dS[:, None, :] / (S ** 2)[:, None, None]
            - what[:, :, None] * ddS[:, None, :] / (S ** 2)[:, None, None]
            + 2.0 * what[:, :, None] * dS[:, None, :] ** 2 / (S ** 3)[:, None, None])
    out = {"what": what, "om": om, "dom": dom, "ddom": ddom, "S": S}
    if with_abs:
        dSa = dwhat_a.sum(axis=1)
        ddSa = ddwhat_a.sum(axis=1)
        out["dom_abs"] = (dwhat_a / S[:, None, None]
                          + what[:, :, None] * dSa[:, None, :] / (S ** 2)[:, None, None])
        out["ddom_abs"] = (ddwhat_a / S[:, None, None]
                           + 2.0 * dwhat_a * dSa[:, None, :] / (S ** 2)[:, None, None]
                           + what[:, :, None] * ddSa[:, None, :] / (S ** 2)[:, None, None]
                           + 2.0 * what[:, :, None] * dSa[:, None, :] ** 2 / (S ** 3)[:, None, None])
    return out


def support_mask(X, level, dim):
    """(n, J_l) boolean: x inside the open support of subdomain j (|theta| < pi in every dimension)."""
    n = level.n
    J = n ** dim
    m = np.ones((X.shape[0], J), dtype=bool)
    for i in range(dim):
        inside = np.abs(X[:, i:i + 1] - level.mu[i][None, :]) < level.sigma[i]
        idx = (np.arange(J) // (n ** i)) % n
        m &= inside[:, idx]
    if getattr(level, "keep", None) is not None:
        m &= level.keep[None, :]
    return m
