"""Least-squares system M a = h of the multilevel ELM-FBPINN (oracle side).

§3 "Definition of vectors" and "Definition of the system matrices":

    f_n     = f(x_n) / sqrt(N_I)
    g_p     = sqrt(lambda_b / N_B^(b)) g_b(x_i^(b))
    N_{n,q} = N[(w_j phi_jk)](x_n) / (sqrt(N_I) L)
    B_{p,q} = sqrt(lambda_b / N_B^(b)) B_b[(w_j phi_jk)](x_i^(b)) / L

with rows stacked interior first, then the boundary sets in order
(Eq. ``multilevel_ls``; p = sum_{m<b} N_B^(m) + i), and columns
q = (level offset) + j K + k (§3 "Indexing conventions").

The operators are applied analytically (reading: the paper does not say how
the derivatives are formed).  For Op[v] = c0 v + sum_i c1_i d_i v +
sum_i c2_i d_ii v and v = w phi the product rule gives

    Op[w phi] = c0 w phi
              + sum_i c1_i (w d_i phi + phi d_i w)
              + sum_i c2_i (w d_ii phi + 2 d_i w d_i phi + phi d_ii w).

Entries are zero outside the support of w_j (§3 "Multilevel
domain-decomposition structure"), so M is stored sparse (CSR) when large.
With the hard-constraint ansatz of §4.3 (problem.ansatz_omega > 0) w is
replaced by A w throughout (oracle/ansatz.py).

Pinned by: the loss identity ||M a - h||^2 = L(a) with the loss of Eq.
``multilevel_loss`` evaluated by finite differences of u_hat; the special cases
J = 1 (w = 1) and w = 0 (phi constant); finite differences of x -> w(x) phi(x)
under each operator (tests/test_oracle_system.py).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.sparse as sp

from .ansatz import ansatz, apply_to_window
from .decomposition import build_levels, n_columns, subdomain_multi_index
from .features import features
from .rng import draw_parameters
from .windows import level_windows, support_mask


@dataclass
class Rows:
    """All rows of the system in the paper's order (interior, then boundary sets)."""
    X: np.ndarray        # (n, d)
    c0: np.ndarray       # (n,)
    c1: np.ndarray       # (n, d)
    c2: np.ndarray       # (n, d)
    scale: np.ndarray    # (n,)  1/sqrt(N_I) or sqrt(lambda_b / N_B^(b))
    rhs: np.ndarray      # (n,)  f or g_b (unscaled)


def stack_rows(problem) -> Rows:
    d = problem.dim
    sets = [problem.interior] + list(problem.boundary)
    X, c0, c1, c2, sc, rhs = [], [], [], [], [], []
    N_I = problem.interior.points.shape[0]
    for s in sets:
        n = s.points.shape[0]
        X.append(np.asarray(s.points, dtype=np.float64).reshape(n, d))
        c0.append(np.full(n, float(s.c0)))
        c1.append(np.tile(np.asarray(s.c1, dtype=np.float64), (n, 1)))
        c2.append(np.tile(np.asarray(s.c2, dtype=np.float64), (n, 1)))
        if s.weight is None:
            sc.append(np.full(n, 1.0 / math.sqrt(N_I)))
        else:
            sc.append(np.full(n, math.sqrt(s.weight / n)))
        rhs.append(np.asarray(s.rhs, dtype=np.float64).reshape(n))
    return Rows(np.concatenate(X), np.concatenate(c0), np.concatenate(c1),
                np.concatenate(c2), np.concatenate(sc), np.concatenate(rhs))


def parameters(problem, round_to_float32: bool = False):
    """Fixed random parameters W, b of every column of the full grids (before
    any subdomain is discarded): row q is full-grid column q."""
    W, b = draw_parameters(problem.seed, problem.n_columns_full, problem.dim,
                           problem.weight_scale)
    if round_to_float32:
        W = W.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    return W, b


def rhs_vector(problem, rows: Optional[np.ndarray] = None) -> np.ndarray:
    R = stack_rows(problem)
    h = R.scale * R.rhs
    return h if rows is None else h[rows]


def assemble(problem, rows: Optional[np.ndarray] = None, fmt: str = "auto",
             with_bound: bool = False, params=None, chunk: int = 8192):
    """Entries of M (and h) for the selected rows (default: all rows).

    fmt: 'dense' (n_rows, N_Phi) array, 'csr' scipy matrix, or 'auto'.
    with_bound: also return 'bound', the same-shaped matrix of
      (scale / L) * [ |c0 w phi| + sum |c1_i| (w |d_i phi| + |phi| |d_i w|_terms)
                      + sum |c2_i| (w |d_ii phi| + 2 |d_i w|_terms |d_i phi| + |phi| |d_ii w|_terms) ],
      the magnitude sum of every product-rule and quotient-rule term, used to
      state rounding tolerances.
    Returns dict(M=..., h=..., bound=...).
    """
    d = problem.dim
    K = problem.features
    R = stack_rows(problem)
    all_rows = np.arange(R.X.shape[0]) if rows is None else np.asarray(rows, dtype=np.int64)
    n_rows = all_rows.shape[0]
    NPhi = n_columns(problem)
    if fmt == "auto":
        fmt = "dense" if n_rows * NPhi <= 6e7 else "csr"
    levels = build_levels(d, problem.lo, problem.hi, problem.levels, problem.delta, K,
                          problem.placement, getattr(problem, "holes", ()))
    L = len(levels)
    W, b = parameters(problem) if params is None else params

    rr, cc, vv, bb = [], [], [], []
    for c_start in range(0, n_rows, chunk):
        sel = all_rows[c_start:c_start + chunk]
        X = R.X[sel]
        c0 = R.c0[sel][:, None]
        c1 = R.c1[sel]
        c2 = R.c2[sel]
        sc = (R.scale[sel] / L)[:, None]
        an = getattr(problem, "ansatz_omega", 0.0)
        if an:
            A, dA, ddA = ansatz(X, problem.lo, problem.hi, an)
        for lev in levels:
            win = level_windows(X, lev, d, with_abs=with_bound)
            mask = support_mask(X, lev, d)
            if an:
                # §4.3: the window factor w becomes g = A w (product rule in A)
                om_, dom_, ddom_ = apply_to_window(A, dA, ddA, win["om"], win["dom"],
                                                   win["ddom"])
                if with_bound:
                    aA = np.abs(A)
                    win["dom_abs"], win["ddom_abs"] = (
                        np.abs(dA)[:, None, :] * win["om"][:, :, None]
                        + aA[:, None, None] * win["dom_abs"],
                        np.abs(ddA)[:, None, :] * win["om"][:, :, None]
                        + 2.0 * np.abs(dA)[:, None, :] * win["dom_abs"]
                        + aA[:, None, None] * win["ddom_abs"])
                win["om"], win["dom"], win["ddom"] = om_, dom_, ddom_
            for j in np.nonzero(mask.any(axis=0))[0]:
                loc = np.nonzero(mask[:, j])[0]
                ji = subdomain_multi_index(lev, d, int(j))
                mu = np.array([lev.mu[i][ji[i]] for i in range(d)])
                sig = np.array(lev.sigma)
                Z = (X[loc] - mu[None, :]) / sig[None, :]
                cols = int(lev.col_first[j]) + np.arange(K)
                pcols = lev.param_offset + int(j) * K + np.arange(K)
                phi, dphi, ddphi, _ = features(Z, W[pcols], b[pcols], sig)
                om = win["om"][loc, j][:, None]
                val = c0[loc] * om * phi
                for i in range(d):
                    dom = win["dom"][loc, j, i][:, None]
                    ddom = win["ddom"][loc, j, i][:, None]
                    val = val + c1[loc, i][:, None] * (om * dphi[:, :, i] + phi * dom)
                    val = val + c2[loc, i][:, None] * (om * ddphi[:, :, i]
                                                       + 2.0 * dom * dphi[:, :, i]
                                                       + phi * ddom)
                val = val * sc[loc]
                rr.append(np.repeat(c_start + loc, K))
                cc.append(np.tile(cols, loc.shape[0]))
                vv.append(val.ravel())
                if with_bound:
                    ap = np.abs(phi)
                    bnd = np.abs(c0[loc]) * om * ap
                    for i in range(d):
                        doma = win["dom_abs"][loc, j, i][:, None]
                        ddoma = win["ddom_abs"][loc, j, i][:, None]
                        adp = np.abs(dphi[:, :, i])
                        bnd = bnd + np.abs(c1[loc, i])[:, None] * (om * adp + ap * doma)
                        bnd = bnd + np.abs(c2[loc, i])[:, None] * (om * np.abs(ddphi[:, :, i])
                                                                   + 2.0 * doma * adp + ap * ddoma)
                    bb.append((bnd * sc[loc]).ravel())

    rows_idx = np.concatenate(rr) if rr else np.zeros(0, np.int64)
    cols_idx = np.concatenate(cc) if cc else np.zeros(0, np.int64)
    vals = np.concatenate(vv) if vv else np.zeros(0)
    out = {"h": (R.scale * R.rhs)[all_rows]}
    if fmt == "dense":
        M = np.zeros((n_rows, NPhi))
        M[rows_idx, cols_idx] = vals
        out["M"] = M
        if with_bound:
            B = np.zeros((n_rows, NPhi))
            B[rows_idx, cols_idx] = np.concatenate(bb)
            out["bound"] = B
    else:
        out["M"] = sp.csr_matrix((vals, (rows_idx, cols_idx)), shape=(n_rows, NPhi))
        if with_bound:
            out["bound"] = sp.csr_matrix((np.concatenate(bb), (rows_idx, cols_idx)),
                                         shape=(n_rows, NPhi))
    return out


def block_max(A: np.ndarray, K: int) -> np.ndarray:
    """Replace every entry of a dense (n, N_Phi) array by the max over its K-column block."""
    n, N = A.shape
    m = np.abs(A).reshape(n, N // K, K).max(axis=2, keepdims=True)
    return np.broadcast_to(m, (n, N // K, K)).reshape(n, N)
