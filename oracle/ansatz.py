"""Hard-constraint ansatz (oracle side).

§4.3 "Hard boundary constraints": the model u_hat is multiplied by

    A(x) = prod_i tanh(w (x_i - lo_i)) tanh(w (hi_i - x_i)),

(the paper writes it for [0,1]^2 with w = omega_{n_omega}), which vanishes on
the boundary of the box, so the boundary loss terms are dropped and the loss
stays quadratic in the coefficients.  The columns of M become
N[A w_j phi_jk] and the product rule gains the derivatives of A:

    g = A w,   d_i g = d_i A w + A d_i w,
    d_ii g = d_ii A w + 2 d_i A d_i w + A d_ii w.

Pinned by: A = 0 on the boundary; central differences of A
(tests/test_oracle_system.py) and of the assembled entries under the
operator.
"""
from __future__ import annotations

import numpy as np


def ansatz(X: np.ndarray, lo, hi, w: float):
    """A, dA (n, d) and ddA (n, d) at points X (n, d); derivatives along each axis."""
    X = np.asarray(X)
    n, d = X.shape
    f = np.ones((n, d), dtype=X.dtype)
    fp = np.zeros((n, d), dtype=X.dtype)
    fpp = np.zeros((n, d), dtype=X.dtype)
    for i in range(d):
        a = np.tanh(w * (X[:, i] - lo[i]))
        b = np.tanh(w * (hi[i] - X[:, i]))
        da = w * (1.0 - a * a)                   # d/dx tanh(w (x - lo))
        db = -w * (1.0 - b * b)                  # d/dx tanh(w (hi - x))
        dda = -2.0 * w * a * da                  # = -2 w^2 a (1 - a^2)
        ddb = 2.0 * w * b * db                   # = -2 w^2 b (1 - b^2)
        f[:, i] = a * b
        fp[:, i] = da * b + a * db
        fpp[:, i] = dda * b + 2.0 * da * db + a * ddb
    A = np.prod(f, axis=1)
    dA = np.zeros((n, d), dtype=X.dtype)
    ddA = np.zeros((n, d), dtype=X.dtype)
    for i in range(d):
        others = np.prod(np.delete(f, i, axis=1), axis=1) if d > 1 else 1.0
        dA[:, i] = fp[:, i] * others
        ddA[:, i] = fpp[:, i] * others
    return A, dA, ddA


def apply_to_window(A, dA, ddA, om, dom, ddom):
    """(g, d_i g, d_ii g) for g = A w, from w and its derivatives at the same points."""
    g = A[:, None] * om
    dg = dA[:, None, :] * om[:, :, None] + A[:, None, None] * dom
    ddg = (ddA[:, None, :] * om[:, :, None] + 2.0 * dA[:, None, :] * dom
           + A[:, None, None] * ddom)
    return g, dg, ddg
