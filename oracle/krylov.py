"""Preconditioned conjugate gradients on the normal equations (oracle side;
not in the paper, which solves with LSQR).

The GPU library also solves M^T M a = M^T h by flexible CG with a block
preconditioner.  With a fixed symmetric positive definite preconditioner,
flexible CG with one kept direction and plain preconditioned CG produce the
same iterates in exact arithmetic, so the oracle is the textbook method
(Hestenes & Stiefel 1952, with a preconditioner):

    r_0 = b - A x_0, z_0 = P r_0, p_0 = z_0;
    alpha_k = r_k.z_k / p_k.A p_k,  x_{k+1} = x_k + alpha_k p_k,
    r_{k+1} = r_k - alpha_k A p_k,  z_{k+1} = P r_{k+1},
    beta_k = r_{k+1}.z_{k+1} / r_k.z_k,  p_{k+1} = z_{k+1} + beta_k p_k.

``block_preconditioner`` builds P: block-Jacobi (the inverse of each K-column
diagonal block of G = M^T M, shifted by eps tr/K), optionally with the first
n_coarse columns (the coarse levels) treated as one joint block shifted by
eps tr/n_coarse -- the coarse-level correction.

``cholesky_dropping`` is the block factorisation with dependent columns
dropped (the GPU's block-Jacobi option drop_tol): an unpivoted Cholesky of
B + eps tr(B)/dim I in column order, where a column whose pivot (its Schur
complement after the earlier kept columns) is at most drop times its shifted
diagonal is dropped -- it takes no part in the factorisation and its
coefficient is fixed at zero.

Pinned by: CG with P = I solves an SPD system in n steps; P = A^{-1} solves it
in one; the joint block over all columns with no shift is A^{-1}; with
drop = 0 the factor is NumPy's Cholesky; a repeated column is dropped and a
Gram of rank r keeps exactly r columns (tests/test_oracle_krylov.py).
"""
from __future__ import annotations

import numpy as np


def pcg(A, b: np.ndarray, P, iters: int, x0: np.ndarray = None) -> np.ndarray:
    """`iters` steps of preconditioned CG; A and P are callables (matrix-vector)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A(x)
    z = P(r)
    p = z.copy()
    rz = r @ z
    for _ in range(iters):
        q = A(p)
        pq = p @ q
        if not pq > 0.0:
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        z = P(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def block_preconditioner(G: np.ndarray, K: int, shift: float, n_coarse: int = 0):
    """z = P r with P = blockdiag(inverse joint coarse block, inverses of the
    K x K diagonal blocks of the finer columns), each block B replaced by
    B + shift tr(B)/dim(B) I before inversion."""
    n = G.shape[0]
    blocks = []
    start = 0
    if n_coarse:
        blocks.append((0, n_coarse))
        start = n_coarse
    for j in range(start, n, K):
        blocks.append((j, min(j + K, n)))
    inv = []
    for a, b in blocks:
        B = 0.5 * (G[a:b, a:b] + G[a:b, a:b].T)
        B = B + shift * np.trace(B) / (b - a) * np.eye(b - a)
        inv.append(np.linalg.inv(B))

    def apply(r):
        z = np.empty_like(r)
        for (a, b), Bi in zip(blocks, inv):
            z[a:b] = Bi @ r[a:b]
        return z
    return apply


def cholesky_dropping(B: np.ndarray, shift: float, drop: float):
    """(L, kept, ratio): L lower triangular with L L^T = the shifted block
    restricted to the kept columns (rows and columns of dropped ones zero),
    kept a bool mask, ratio[k] the pivot of column k over its shifted
    diagonal when its turn came."""
    n = B.shape[0]
    S = 0.5 * (B + B.T) + shift * np.trace(B) / n * np.eye(n)
    g = np.diag(S).copy()          # the shifted diagonal, the drop test's scale
    L = np.zeros((n, n))
    kept = np.ones(n, dtype=bool)
    ratio = np.zeros(n)
    for k in range(n):
        d = S[k, k]
        ratio[k] = d / g[k]
        if drop > 0.0 and not d > drop * g[k]:
            kept[k] = False        # dependent on the kept columns before it
            continue
        if not d > 0.0:
            raise np.linalg.LinAlgError("non-positive pivot")
        col = S[k:, k] / np.sqrt(d)
        L[k:, k] = col
        S[k + 1:, k + 1:] -= np.outer(col[1:], col[1:])
    L[~kept, :] = 0.0              # a dropped row takes no part either
    return L, kept, ratio
