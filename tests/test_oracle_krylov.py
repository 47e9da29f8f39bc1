"""Pins of the oracle's preconditioned CG and block preconditioner."""
import numpy as np

from oracle import krylov as KR


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(np.linspace(1.0, 50.0, n)) @ Q.T


def test_cg_solves_spd_system_in_n_steps():
    A = _spd(12, 0)
    b = np.random.default_rng(1).standard_normal(12)
    x = KR.pcg(lambda v: A @ v, b, lambda r: r, 12)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def test_exact_preconditioner_solves_in_one_step():
    A = _spd(10, 2)
    b = np.random.default_rng(3).standard_normal(10)
    Ai = np.linalg.inv(A)
    x = KR.pcg(lambda v: A @ v, b, lambda r: Ai @ r, 1)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_joint_block_over_every_column_is_the_inverse():
    A = _spd(9, 4)
    P = KR.block_preconditioner(A, K=3, shift=0.0, n_coarse=9)
    r = np.random.default_rng(5).standard_normal(9)
    assert np.allclose(P(r), np.linalg.solve(A, r), rtol=1e-10)


def test_block_jacobi_blocks_and_shift():
    """Without a coarse block: each K-block is inverted on its own, shifted by
    eps tr/K (written out for a 2 x 2 block)."""
    A = _spd(6, 6)
    eps = 0.1
    P = KR.block_preconditioner(A, K=2, shift=eps)
    r = np.zeros(6)
    r[2] = 1.0
    B = A[2:4, 2:4] + eps * np.trace(A[2:4, 2:4]) / 2 * np.eye(2)
    z = P(r)
    assert np.allclose(z[2:4], np.linalg.solve(B, [1.0, 0.0]))
    assert np.all(z[:2] == 0.0) and np.all(z[4:] == 0.0)


def test_cholesky_dropping_without_drop_is_cholesky():
    A = _spd(8, 7)
    L, kept, _ = KR.cholesky_dropping(A, 1e-3, 0.0)
    assert kept.all()
    ref = np.linalg.cholesky(A + 1e-3 * np.trace(A) / 8 * np.eye(8))
    assert np.allclose(L, ref, rtol=1e-12, atol=1e-14)


def test_cholesky_dropping_drops_a_repeated_column():
    """Column 3 repeats column 1: its Schur complement is the shift alone
    (1e-10 of the mean diagonal), far below a 1e-6 drop ratio; the factor of
    the kept columns is the Cholesky of their own shifted block."""
    rng = np.random.default_rng(8)
    M = rng.standard_normal((30, 5))
    M[:, 3] = M[:, 1]
    B = M.T @ M
    L, kept, ratio = KR.cholesky_dropping(B, 1e-10, 1e-6)
    assert kept.tolist() == [True, True, True, False, True]
    assert ratio[3] < 1e-9 < ratio[[0, 1, 2, 4]].min()
    sub = np.ix_(kept, kept)
    Bs = B + 1e-10 * np.trace(B) / 5 * np.eye(5)
    assert np.allclose(L[sub] @ L[sub].T, Bs[sub], rtol=1e-10)
    assert np.all(L[3, :] == 0.0) and np.all(L[:, 3] == 0.0)


def test_cholesky_dropping_keeps_the_rank():
    """A Gram of rank 6 in dimension 10 (10 features, 6 points, in general
    position) keeps exactly its first 6 columns."""
    rng = np.random.default_rng(9)
    M = rng.standard_normal((6, 10))
    _, kept, _ = KR.cholesky_dropping(M.T @ M, 1e-12, 1e-8)
    assert kept.tolist() == [True] * 6 + [False] * 4
