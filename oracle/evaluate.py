"""Evaluation of the trained model and the paper's error metric (oracle side).

* ``u_hat``  Eq. ``multilevel_solution``:
             u_hat(x) = (1/L) sum_l sum_j w_j(x) sum_k a_ljk phi_ljk(x),
             times A(x) under the hard-constraint ansatz of §4.3
* ``e_l1``   Eq. ``l1_error``: sum_i |u_hat(x_i) - u(x_i)| / (M * std(u)),
             std taken over the test set with the population convention
             (reading: the paper does not say which).
* ``rel_l2`` ||u_hat - u||_2 / ||u||_2 over the test points.

Pinned by: u_hat equals M a for the identity operator with unit row scale
(the c0 = 1 column of the assembly), exact reproduction of a function in the
span, and the closed-form value of e_l1 on a hand-made example
(tests/test_oracle_evaluate.py).
"""
from __future__ import annotations

import numpy as np

from .ansatz import ansatz
from .decomposition import build_levels, subdomain_multi_index
from .features import features
from .system import parameters
from .windows import level_windows, support_mask


def u_hat(problem, a: np.ndarray, X: np.ndarray, params=None, chunk: int = 8192) -> np.ndarray:
    d = problem.dim
    K = problem.features
    levels = build_levels(d, problem.lo, problem.hi, problem.levels, problem.delta, K,
                          problem.placement, getattr(problem, "holes", ()))
    L = len(levels)
    W, b = parameters(problem) if params is None else params
    X = np.asarray(X, dtype=np.float64).reshape(-1, d)
    out = np.zeros(X.shape[0])
    for c_start in range(0, X.shape[0], chunk):
        Xc = X[c_start:c_start + chunk]
        acc = np.zeros(Xc.shape[0])
        for lev in levels:
            win = level_windows(Xc, lev, d)
            mask = support_mask(Xc, lev, d)
            for j in np.nonzero(mask.any(axis=0))[0]:
                loc = np.nonzero(mask[:, j])[0]
                ji = subdomain_multi_index(lev, d, int(j))
                mu = np.array([lev.mu[i][ji[i]] for i in range(d)])
                sig = np.array(lev.sigma)
                cols = int(lev.col_first[j]) + np.arange(K)
                pcols = lev.param_offset + int(j) * K + np.arange(K)
                phi, _, _, _ = features((Xc[loc] - mu) / sig, W[pcols], b[pcols], sig)
                acc[loc] += win["om"][loc, j] * (phi @ a[cols])
        out[c_start:c_start + chunk] = acc / L
        an = getattr(problem, "ansatz_omega", 0.0)
        if an:      # §4.3: the model is A(x) u_hat(x)
            out[c_start:c_start + chunk] *= ansatz(Xc, problem.lo, problem.hi, an)[0]
    return out


def e_l1(uh: np.ndarray, u: np.ndarray) -> float:
    u = np.asarray(u, dtype=np.float64)
    return float(np.sum(np.abs(uh - u)) / (u.size * np.std(u)))


def rel_l2(uh: np.ndarray, u: np.ndarray) -> float:
    u = np.asarray(u, dtype=np.float64)
    return float(np.linalg.norm(uh - u) / np.linalg.norm(u))
