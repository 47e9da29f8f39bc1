"""Least-squares minimiser of ||M a - h|| (oracle side).

The method's result is the minimiser of Eq. ``multilevel_ls``; the paper
reaches it with SciPy's LSQR (§3 last paragraph, §4.1 "Optimisation and
solvers": at most 15000 iterations, run to the full budget).  M is numerically
rank deficient (the paper reports condition numbers up to ~1e20), so several
minimisers exist and only u_hat and the residual are compared, never a.

* ``lstsq_qr``   the plain definition for sizes that fit dense: Householder QR
                 with column pivoting (LAPACK geqp3 through scipy), rank cut
                 |R_kk| <= rcond |R_11|, basic solution by back substitution.
* ``lstsq_lsqr`` the paper's own route (SciPy LSQR, Paige & Saunders 1982) for
                 systems too large for dense QR.

Pinned by: agreement with an SVD pseudo-inverse solve on tiny full-rank
problems, exact recovery of a planted coefficient vector (residual ~ 0),
orthogonality M^T (M a - h) ~ 0 (tests/test_oracle_lstsq.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def lstsq_qr(M: np.ndarray, h: np.ndarray, rcond: float = 1e-13):
    """Basic least-squares solution by column-pivoted Householder QR.

    Returns (a, rank).
    """
    M = np.asarray(M, dtype=np.float64)
    Q, R, P = sla.qr(M, mode="economic", pivoting=True)
    diag = np.abs(np.diag(R))
    if diag.size == 0 or diag[0] == 0.0:
        return np.zeros(M.shape[1]), 0
    rank = int(np.count_nonzero(diag > rcond * diag[0]))
    y = Q.T @ h
    z = sla.solve_triangular(R[:rank, :rank], y[:rank], lower=False)
    a = np.zeros(M.shape[1])
    a[P[:rank]] = z
    return a, rank


def _row_split_operator(M, threads: int):
    """M as a LinearOperator whose products run on row blocks in threads.

    Each output entry is the same CSR row sum as in the serial product (rows
    of M for M x, rows of the CSR transpose for M^T y), so results are
    bitwise those of the serial SciPy product.
    """
    from concurrent.futures import ThreadPoolExecutor
    M = sp.csr_matrix(M)
    MT = M.T.tocsr()
    ex = ThreadPoolExecutor(threads)

    def parts(A):
        b = np.linspace(0, A.shape[0], threads + 1).astype(np.int64)
        return [(b[i], b[i + 1], A[b[i]:b[i + 1]]) for i in range(threads)]

    pm, pt = parts(M), parts(MT)

    def apply(ps, v, n):
        out = np.empty(n)

        def one(p):
            out[p[0]:p[1]] = p[2] @ v
        list(ex.map(one, ps))
        return out

    return spla.LinearOperator(M.shape, matvec=lambda v: apply(pm, v, M.shape[0]),
                               rmatvec=lambda v: apply(pt, v, M.shape[1]), dtype=np.float64)


def lstsq_lsqr(M, h: np.ndarray, iter_lim: int = 15000, atol: float = 0.0, btol: float = 0.0,
               threads: int = 1):
    """SciPy LSQR, by default run for the full iteration budget as in the paper.

    threads > 1 runs the matrix products on row blocks in threads (same values).
    Returns (a, info) with info = dict(istop, itn, r1norm, arnorm).
    """
    if not sp.issparse(M):
        M = sp.csr_matrix(M)
    A = _row_split_operator(M, threads) if threads > 1 else M
    res = spla.lsqr(A, h, atol=atol, btol=btol, conlim=0.0, iter_lim=iter_lim)
    a, istop, itn, r1norm = res[0], res[1], res[2], res[3]
    return a, {"istop": int(istop), "itn": int(itn), "r1norm": float(r1norm),
               "arnorm": float(res[7])}


def residual_norms(M, a: np.ndarray, h: np.ndarray):
    """(||M a - h||, ||M^T (M a - h)||)."""
    r = M @ a - h
    return float(np.linalg.norm(r)), float(np.linalg.norm(M.T @ r))
