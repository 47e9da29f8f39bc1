"""Least-squares minimiser of ||M a - h|| (oracle side).

The method's result is the minimiser of Eq. ``multilevel_ls``; the paper
reaches it with SciPy's LSQR (§3 last paragraph, §4.1 "Optimisation and
solvers": at most 15000 iterations, run to the full budget).  M is numerically
rank deficient (the paper reports condition numbers up to ~1e20), so several
minimisers exist and only u_hat and the residual are compared, never a.

* ``lstsq_qr``   the plain definition for sizes that fit dense: the project's
                 own Householder QR with column pivoting (Businger & Golub
                 1965; Golub & Van Loan, "Matrix Computations", QR with column
                 pivoting), no LAPACK.  Each step takes the remaining column of
                 largest norm, stops once that norm is <= rcond |R_11| (the
                 rank cut), and the basic solution follows by back substitution.
* ``lstsq_lsqr`` the paper's own route (SciPy LSQR, Paige & Saunders 1982) for
                 systems too large for dense QR.
* ``golub_kahan`` k steps of the Golub-Kahan bidiagonalisation that LSQR runs
                 (Paige & Saunders 1982, their §3): the alpha and beta that give
                 the singular-value (condition number) estimates of M.

Pinned by (tests/test_oracle_lstsq.py): planted rank-deficient systems whose
rank, residual norm and fitted values are known in closed form; an upper
triangular system that needs no pivoting; orthogonal columns whose pivot order
and R diagonal are their norms; the normal equations; exact recovery of a
planted coefficient vector on an assembled system; the bidiagonal of a
diagonal matrix and the full-length bidiagonal's singular values.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _column_blocks(n0: int, n: int, width: int = 512):
    return [(s, min(s + width, n)) for s in range(n0, n, width)]


def qr_pivoted(M: np.ndarray, h: np.ndarray, rcond: float = 1e-13, threads: int = 1):
    """Householder QR with column pivoting of [M | h], h never pivoted.

    Step k: take the column of largest Euclidean norm over rows k.. among the
    columns not yet taken (the first such column on ties); if that norm is
    <= rcond times the first step's, stop (rank = k).  Otherwise swap it into
    place, reflect rows k.. by H = I - 2 v v^T / (v^T v) with v = x - beta e_1,
    beta = -sign(x_1) ||x|| (so R_kk = beta), apply H to every later column
    and to h, and recompute the later columns' norms over rows k+1.. exactly.

    Returns (R [rank x rank] upper triangular, Q^T h [rank], perm [n], rank):
    column perm[i] of M is the i-th pivot.  threads > 1 splits the column
    updates over threads (the same arithmetic per column).
    """
    A = np.array(M, dtype=np.float64, order="F", copy=True)
    y = np.array(h, dtype=np.float64, copy=True)
    m, n = A.shape
    perm = np.arange(n)
    cn = np.einsum("ij,ij->j", A, A)         # squared column norms over rows 0..
    pool = ThreadPoolExecutor(threads) if threads > 1 else None
    r11 = 0.0
    rank = 0
    for k in range(min(m, n)):
        j = k + int(np.argmax(cn[k:]))
        rkk = np.sqrt(cn[j])
        if k == 0:
            r11 = rkk
        if rkk == 0.0 or rkk <= rcond * r11:
            break
        if j != k:
            A[:, [k, j]] = A[:, [j, k]]
            cn[[k, j]] = cn[[j, k]]
            perm[[k, j]] = perm[[j, k]]
        x = A[k:, k].copy()
        beta = -np.copysign(np.linalg.norm(x), x[0])
        v = x
        v[0] -= beta
        c = 2.0 / (v @ v)
        A[k, k] = beta
        A[k + 1:, k] = 0.0

        def update(block):
            s, e = block
            B = A[k:, s:e]
            B -= np.outer(c * v, v @ B)
            cn[s:e] = np.einsum("ij,ij->j", B[1:], B[1:])

        blocks = _column_blocks(k + 1, n)
        if pool is not None:
            list(pool.map(update, blocks))
        else:
            for b in blocks:
                update(b)
        y[k:] -= (c * (v @ y[k:])) * v
        rank = k + 1
    if pool is not None:
        pool.shutdown()
    R = np.triu(A[:rank, :rank])
    return R, y[:rank].copy(), perm, rank


def back_substitute(R: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Solve R z = y for upper triangular R, last row first."""
    r = R.shape[0]
    z = np.zeros(r)
    for i in range(r - 1, -1, -1):
        z[i] = (y[i] - R[i, i + 1:] @ z[i + 1:]) / R[i, i]
    return z


def lstsq_qr(M: np.ndarray, h: np.ndarray, rcond: float = 1e-13, threads: int = 1):
    """Basic least-squares solution by column-pivoted Householder QR.

    a[perm[i]] = z[i] for the retained pivots, 0 elsewhere.  Returns (a, rank).
    """
    M = np.asarray(M, dtype=np.float64)
    R, y, perm, rank = qr_pivoted(M, h, rcond, threads)
    a = np.zeros(M.shape[1])
    if rank:
        a[perm[:rank]] = back_substitute(R, y)
    return a, rank


def golub_kahan(M, h: np.ndarray, k: int):
    """k steps of the Golub-Kahan bidiagonalisation started from h.

    beta_1 u_1 = h, alpha_1 v_1 = M^T u_1, then for i = 1..k
    beta_{i+1} u_{i+1} = M v_i - alpha_i u_i and
    alpha_{i+1} v_{i+1} = M^T u_{i+1} - beta_{i+1} v_i (no reorthogonalisation,
    as in LSQR).  Returns (alpha [k], beta [k+1]): the lower bidiagonal
    B_k ((k+1) x k) has alpha on its diagonal and beta_2..beta_{k+1} below it.
    """
    beta = [float(np.linalg.norm(h))]
    u = h / beta[0]
    v = M.T @ u
    alpha = [float(np.linalg.norm(v))]
    v = v / alpha[0]
    for i in range(k):
        u = M @ v - alpha[i] * u
        beta.append(float(np.linalg.norm(u)))
        u = u / beta[-1]
        if i + 1 == k:
            break
        v = M.T @ u - beta[-1] * v
        alpha.append(float(np.linalg.norm(v)))
        v = v / alpha[-1]
    return np.array(alpha), np.array(beta)


def bidiagonal(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """The (k+1) x k lower bidiagonal B_k of Golub-Kahan."""
    k = alpha.size
    B = np.zeros((k + 1, k))
    B[np.arange(k), np.arange(k)] = alpha
    B[np.arange(1, k + 1), np.arange(k)] = beta[1:k + 1]
    return B


def _row_split_operator(M, threads: int):
    """M as a LinearOperator whose products run on row blocks in threads.

    Each output entry is the same CSR row sum as in the serial product (rows
    of M for M x, rows of the CSR transpose for M^T y), so results are
    bitwise those of the serial SciPy product.
    """
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
