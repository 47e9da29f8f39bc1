"""Pins of the oracle's least-squares solvers (Eq. multilevel_ls).

The QR solver is the project's own column-pivoted Householder QR; it is
pinned to systems whose answer is known in closed form (planted rank,
residual and fitted values; triangular and orthogonal-column systems), to
the normal equations, and to exact recovery on an assembled system.  LSQR is
SciPy's (the paper's solver).  The Golub-Kahan bidiagonalisation is pinned to
a diagonal matrix (closed form) and to the singular values of M.
"""
import numpy as np
import pytest

import workloads as WL
from oracle import evaluate as E
from oracle import lstsq as LS
from oracle import system as S


def _orthonormal(m, n, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, n)))
    return Q


def test_planted_rank_deficient_system():
    """A = [Q D, Q D C]: rank r, range = span(Q); h = Q g + r_perp with r_perp
    orthogonal to range(A), so the minimal residual is r_perp and the fitted
    values are Q g exactly, whatever basic solution is taken."""
    m, r = 40, 5
    Qfull = _orthonormal(m, r + 1, 3)
    Q, q_perp = Qfull[:, :r], Qfull[:, r]
    D = np.diag([3.0, 2.0, 1.5, 1.0, 0.5])
    C = np.random.default_rng(4).standard_normal((r, 4))
    A = np.hstack([Q @ D, Q @ D @ C])
    g = np.array([1.0, -2.0, 0.5, 3.0, -1.0])
    h = Q @ g + 0.7 * q_perp
    a, rank = LS.lstsq_qr(A, h)
    assert rank == r
    res = A @ a - h
    assert np.linalg.norm(res) == pytest.approx(0.7, rel=1e-12)
    assert np.allclose(A @ a, Q @ g, atol=1e-12)
    assert np.count_nonzero(a) == r            # a basic solution: r nonzeros


def test_upper_triangular_needs_no_pivoting():
    """Columns already ordered by decreasing norm with R = A: the solution is
    the back substitution of the printed triangle."""
    R = np.array([[4.0, 1.0, -1.0],
                  [0.0, 3.0, 0.5],
                  [0.0, 0.0, 2.0]])
    h = np.array([1.0, 2.0, 4.0])
    a, rank = LS.lstsq_qr(R, h)
    assert rank == 3
    # z3 = 2, z2 = (2 - 0.5*2)/3 = 1/3, z1 = (1 - 1/3 + 2)/4 = 2/3
    assert np.allclose(a, [2.0 / 3.0, 1.0 / 3.0, 2.0], rtol=0, atol=1e-15)


def test_orthogonal_columns_pivot_by_norm():
    """Orthogonal columns of norms 1, 5, 1e-15, 2: pivots in norm order, the
    1e-15 column falls under the rank cut, R's diagonal magnitudes are the
    norms and each coefficient is the projection of h on its column."""
    Q = _orthonormal(10, 4, 5)
    norms = np.array([1.0, 5.0, 1e-15, 2.0])
    A = Q * norms
    h = np.random.default_rng(6).standard_normal(10)
    R, y, perm, rank = LS.qr_pivoted(A, h)
    assert rank == 3
    assert list(perm[:3]) == [1, 3, 0]
    assert np.allclose(np.abs(np.diag(R)), [5.0, 2.0, 1.0], rtol=1e-14)
    a, _ = LS.lstsq_qr(A, h)
    assert np.allclose(a[[0, 1, 3]], (Q.T @ h)[[0, 1, 3]] / norms[[0, 1, 3]], rtol=1e-12)
    assert a[2] == 0.0


def test_full_rank_solution_satisfies_normal_equations():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((60, 12))
    h = rng.standard_normal(60)
    a, rank = LS.lstsq_qr(A, h)
    assert rank == 12
    # the normal equations, solved by Gaussian elimination: another route
    ref = np.linalg.solve(A.T @ A, A.T @ h)
    assert np.allclose(a, ref, rtol=1e-10, atol=1e-12)
    assert np.linalg.norm(A.T @ (A @ a - h)) <= 1e-12 * np.linalg.norm(A) ** 2 * np.linalg.norm(a)


def test_threaded_qr_is_bitwise_serial():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((300, 1200)) @ np.diag(np.exp(-np.linspace(0, 30, 1200)))
    h = rng.standard_normal(300)
    a1, r1 = LS.lstsq_qr(A, h)
    a4, r4 = LS.lstsq_qr(A, h, threads=4)
    assert r1 == r4 and np.array_equal(a1, a4)


def test_lsqr_matches_qr_on_well_conditioned_problem():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((80, 20)) + 3 * np.eye(80, 20)
    h = rng.standard_normal(80)
    a1, _ = LS.lstsq_qr(A, h)
    a2, info = LS.lstsq_lsqr(A, h, iter_lim=500, atol=1e-15, btol=1e-15)
    assert np.allclose(a1, a2, rtol=1e-9, atol=1e-10)


def test_exact_recovery_of_planted_solution():
    """rhs generated from a planted coefficient vector: residual ~ 0 and u_hat reproduced."""
    P = WL.dho(levels=(1, 2), features=6, n_interior=200, omega0=6.0, seed=4)
    out = S.assemble(P, fmt="dense")
    M = out["M"]
    rng = np.random.default_rng(5)
    a_star = rng.standard_normal(P.n_columns)
    h = M @ a_star
    a, rank = LS.lstsq_qr(M, h)
    assert np.linalg.norm(M @ a - h) <= 1e-9 * np.linalg.norm(h)
    X = P.test_points
    u_star = E.u_hat(P, a_star, X)
    assert np.allclose(E.u_hat(P, a, X), u_star, atol=1e-6 * np.abs(u_star).max())


def test_golub_kahan_of_diagonal_matrix():
    """M = diag(d) (square), h = ones: alpha_1 = ||d|| / sqrt(n) and
    beta_2 = the norm of d*d/||d|| - alpha_1 u_1 (the first Lanczos step,
    written out by hand)."""
    d = np.array([1.0, 2.0, 3.0, 4.0])
    M = np.diag(d)
    h = np.ones(4)
    al, be = LS.golub_kahan(M, h, 1)
    assert be[0] == pytest.approx(2.0)
    u1 = h / 2.0
    assert al[0] == pytest.approx(np.linalg.norm(d) / 2.0, rel=1e-15)
    v1 = d / np.linalg.norm(d)
    assert be[1] == pytest.approx(np.linalg.norm(d * v1 - al[0] * u1), rel=1e-14)


def test_golub_kahan_full_length_reproduces_singular_values():
    """After n steps on a well-conditioned n-column M (h with components in
    every singular direction) the bidiagonal's singular values are M's."""
    rng = np.random.default_rng(9)
    U = _orthonormal(30, 6, 10)
    V = _orthonormal(6, 6, 11)
    sv = np.array([5.0, 3.0, 2.0, 1.5, 1.0, 0.5])
    M = U @ np.diag(sv) @ V.T
    h = U @ rng.standard_normal(6) + 0.1 * rng.standard_normal(30)
    al, be = LS.golub_kahan(M, h, 6)
    B = LS.bidiagonal(al, be)
    got = np.linalg.svd(B, compute_uv=False)
    assert np.allclose(np.sort(got), np.sort(sv), rtol=1e-10)


def test_threaded_lsqr_is_bitwise_serial():
    P = WL.dho(levels=(1, 2, 4), features=8, n_interior=300, omega0=8.0)
    out = S.assemble(P, fmt="csr")
    a1, _ = LS.lstsq_lsqr(out["M"], out["h"], iter_lim=200)
    a4, _ = LS.lstsq_lsqr(out["M"], out["h"], iter_lim=200, threads=4)
    assert np.array_equal(a1, a4)
