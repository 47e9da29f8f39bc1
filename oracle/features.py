"""Shallow random tanh features (oracle side).

§3 Eq. (shallow networks) with h = 1 hidden layer and Xi = tanh: each column
(l, j, k) is phi(x) = tanh(w . z + b) with fixed random w, b.  Readings:

* z is the subdomain-normalised input z = (x - mu_j) / sigma_j (the FBPINN
  convention of normalising each subdomain network's input; the scaled-input
  reading of the workload definitions);
* a bias b is included (§4.1 initialises W and b; without it every feature is
  odd about the centre and the local basis is degenerate).

Derivatives w.r.t. x_i follow from the chain rule with ds/dx_i = w_i / sigma_i:
    d_i phi  = (1 - phi^2) w_i / sigma_i
    d_ii phi = -2 phi (1 - phi^2) (w_i / sigma_i)^2

Pinned by central finite differences and complex-step derivatives of
x -> tanh(w.(x - mu)/sigma + b) (tests/test_oracle_features.py).
"""
from __future__ import annotations

import numpy as np


def features(Z, W, b, sigma):
    """Features of one subdomain at normalised points Z.

    Z: (n, d) normalised coordinates; W: (K, d); b: (K,); sigma: (d,).
    Returns phi (n, K), dphi (n, K, d), ddphi (n, K, d), s (n, K).
    """
    s = Z @ W.T + b[None, :]
    phi = np.tanh(s)
    t = 1.0 - phi * phi
    wt = W / np.asarray(sigma)[None, :]          # ds/dx_i, (K, d)
    dphi = t[:, :, None] * wt[None, :, :]
    ddphi = (-2.0 * phi * t)[:, :, None] * (wt * wt)[None, :, :]
    return phi, dphi, ddphi, s
