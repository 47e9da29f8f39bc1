"""GPU condition-number and rank diagnostics against the oracle.

The paper reports kappa(M) in every results table (§4) and discusses the
numerical rank of M (§5).  The library estimates both on the device:

* LSQR records its Golub-Kahan bidiagonalisation (Paige & Saunders 1982, §3),
  alpha_1.., beta_1..; the extreme singular values of the lower bidiagonal
  B_k bound those of the operator from inside (sigma_max(B_k) <= sigma_max,
  sigma_min(B_k) >= sigma_min), so kappa(B_k) is a lower bound of kappa that
  grows with k.  They are found by Sturm-count bisection of B_k's
  Golub-Kahan tridiagonal in one warp.
* The QR solve reports its numerical rank and |R_11|, |R_rr|.

The GPU's alpha and beta are compared with the oracle's own bidiagonalisation
of the same M, and its extreme singular values with NumPy's SVD of the
oracle's B_k; the QR rank with the oracle's.
"""
import numpy as np
import pytest

import paper_2409_01949_gb300 as E
import workloads as WL
from oracle import lstsq as OL
from oracle import system as OS

pytestmark = pytest.mark.gpu


def _small():
    return WL.poisson1d(levels=(4,), features=4, n_interior=200, lam=100.0)


@pytest.mark.parametrize("prec", [E.FP64, E.DF32])
def test_lsqr_bidiagonal_matches_oracle_golub_kahan(prec):
    """Plain LSQR (no preconditioner) for k = 6 steps: alpha_1..alpha_7 and
    beta_1..beta_7 equal the oracle's (Lanczos rounding stays below 1e-12 at
    k = 6 on this kappa ~ 8e3 system)."""
    P = _small()
    ref = OS.assemble(P, fmt="dense")
    k = 6
    al_o, be_o = OL.golub_kahan(ref["M"], ref["h"], k + 1)
    with E.Solver.from_problem(P, precision=prec) as s:
        s.assemble_problem(P)
        info = s.solve(preconditioner=E.PREC_NONE, max_iter=k, atol=0.0, btol=0.0,
                       check_every=1)
        al, be = s.bidiagonal()
    assert info.iterations == k and al.size == k + 1 and be.size == k + 1
    tol = 1e-12 if prec == E.FP64 else 1e-11
    assert np.allclose(al, al_o[:k + 1], rtol=tol, atol=0)
    assert np.allclose(be, be_o[:k + 1], rtol=tol, atol=0)


def test_extreme_singular_values_of_bidiagonal():
    """sigma_max and sigma_min reported by the solve equal NumPy's SVD of the
    (k+1) x k bidiagonal built from the GPU's own alpha, beta, for k = 3, 12
    and 40 (the last past where sigma_min has settled), to the bisection's
    1e-10 relative width."""
    P = _small()
    for k in (3, 12, 40):
        with E.Solver.from_problem(P, precision=E.FP64) as s:
            s.assemble_problem(P)
            info = s.solve(preconditioner=E.PREC_NONE, max_iter=k, atol=0.0, btol=0.0,
                           check_every=k)
            al, be = s.bidiagonal()
        sv = np.linalg.svd(OL.bidiagonal(al[:k], be[:k + 1]), compute_uv=False)
        print(k, info.sigma_max, sv.max(), info.sigma_min, sv.min())
        # the bisection stops at 1e-10 relative width
        assert info.sigma_max == pytest.approx(sv.max(), rel=1e-10)
        assert info.sigma_min == pytest.approx(sv.min(), rel=1e-9)


def test_condition_estimate_grows_towards_kappa_of_M():
    """On the full-rank 16-column system, kappa(B_k) never exceeds kappa(M)
    (NumPy SVD of the oracle's M), does not decrease with k, and reaches it
    (to 1e-6) by k = 64.  Without reorthogonalisation the Lanczos vectors lose
    orthogonality, so 16 steps are not enough: the oracle's own
    bidiagonalisation gives kappa(B_16) = 355 and kappa(B_32) = 8491.24 against
    kappa(M) = 8491.25."""
    P = _small()
    M = OS.assemble(P, fmt="dense")["M"]
    sv = np.linalg.svd(M, compute_uv=False)
    kappa = sv[0] / sv[-1]
    prev = 0.0
    for k in (2, 4, 8, 16, 32, 64):
        with E.Solver.from_problem(P, precision=E.FP64) as s:
            s.assemble_problem(P)
            info = s.solve(preconditioner=E.PREC_NONE, max_iter=k, atol=0.0, btol=0.0,
                           check_every=k)
        est = info.sigma_max / info.sigma_min
        print(f"k={k}: kappa(B_k) {est:.4e}, kappa(M) {kappa:.4e}")
        assert est <= kappa * (1 + 1e-8)
        assert est >= prev * (1 - 1e-12)
        prev = est
    assert prev == pytest.approx(kappa, rel=1e-6)


def test_qr_rank_and_r11_match_oracle():
    """QR on the multilevel DHO system: numerical rank within 1 of the
    oracle's, |R_11| (the largest column norm) equal to the oracle's, and
    |R_rr| on the kept side of the rank cut (> 1e-13 |R_11|)."""
    P = WL.dho(levels=(1, 2, 4), features=16, n_interior=300, omega0=10.0)
    ref = OS.assemble(P, fmt="dense")
    R, _, _, rank = OL.qr_pivoted(ref["M"], ref["h"])
    with E.Solver.from_problem(P, precision=E.FP64) as s:
        s.assemble_problem(P)
        info = s.solve(method=E.SOLVE_QR)
    assert abs(info.rank - rank) <= 1
    assert info.sigma_max == pytest.approx(abs(R[0, 0]), rel=1e-13)
    assert 1e-13 * info.sigma_max < info.sigma_min <= info.sigma_max
