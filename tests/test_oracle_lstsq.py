"""Pins of the oracle's least-squares solvers (Eq. multilevel_ls)."""
import numpy as np
import pytest

import workloads as WL
from oracle import evaluate as E
from oracle import lstsq as LS
from oracle import system as S


def test_qr_matches_svd_solution_on_full_rank_problem():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((60, 12))
    h = rng.standard_normal(60)
    a, rank = LS.lstsq_qr(A, h)
    ref = np.linalg.lstsq(A, h, rcond=None)[0]      # SVD-based (LAPACK gelsd), another route
    assert rank == 12
    assert np.allclose(a, ref, rtol=1e-11, atol=1e-12)


def test_lsqr_matches_qr_on_well_conditioned_problem():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((80, 20)) + 3 * np.eye(80, 20)
    h = rng.standard_normal(80)
    a1, _ = LS.lstsq_qr(A, h)
    a2, info = LS.lstsq_lsqr(A, h, iter_lim=500, atol=1e-15, btol=1e-15)
    assert np.allclose(a1, a2, rtol=1e-9, atol=1e-10)


def test_rank_deficient_basic_solution_minimises_residual():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((50, 6))
    A = np.hstack([B, B[:, :3] @ rng.standard_normal((3, 4))])   # rank 6 of 10 columns
    h = rng.standard_normal(50)
    a, rank = LS.lstsq_qr(A, h)
    assert rank == 6
    r = A @ a - h
    ref = A @ np.linalg.lstsq(A, h, rcond=None)[0] - h
    assert np.linalg.norm(r) == pytest.approx(np.linalg.norm(ref), rel=1e-12)
    assert np.linalg.norm(A.T @ r) <= 1e-10 * np.linalg.norm(A) * np.linalg.norm(r)


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


def test_threaded_lsqr_is_bitwise_serial():
    P = WL.dho(levels=(1, 2, 4), features=8, n_interior=300, omega0=8.0)
    out = S.assemble(P, fmt="csr")
    a1, _ = LS.lstsq_lsqr(out["M"], out["h"], iter_lim=200)
    a4, _ = LS.lstsq_lsqr(out["M"], out["h"], iter_lim=200, threads=4)
    assert np.array_equal(a1, a4)
