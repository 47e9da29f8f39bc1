"""Edge and degenerate cases of the GPU path against the oracle.

* h = 0 (f and g zero): the least-squares minimiser is a = 0; LSQR's first
  Golub-Kahan step has beta_1 = 0 and the solve returns zeros, finite, without
  iterating on FP32 panels (the device's stopping test) and within the first
  check on FP64 panels.
* Evaluation at no points returns an empty result.
* K = 160, past the fused pass's 128 features: LSQR takes the general
  (gather / transpose) path, whose first iterates equal SciPy's on the
  oracle's M; block-Jacobi, built for K <= 128, reports ERR_UNSUPPORTED.
* An empty batch is a no-op.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import paper_2409_01949_gb300 as E
import workloads as WL
from oracle import system as OS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [E.FP32, E.FP64])
def test_zero_right_hand_side_gives_zero_coefficients(prec):
    P = WL.poisson2d(levels=(1, 2, 4), features=32, n_side=30, n_boundary_side=30)
    sets = [dict(points=np.ascontiguousarray(rs.points, dtype=np.float64),
                 rhs=np.zeros(rs.points.shape[0]), c0=rs.c0, c1=rs.c1, c2=rs.c2,
                 weight=rs.weight) for rs in [P.interior] + list(P.boundary)]
    with E.Solver.from_problem(P, precision=prec) as s:
        s.assemble(sets)
        info = s.solve(max_iter=100, atol=0.0, btol=0.0, ntol=1e-6, shift=1e-6,
                       check_every=10)
        a = s.coeffs()
    assert info.status == E.OK
    assert np.all(a == 0.0)
    if prec == E.FP32:
        assert info.iterations == 0
    else:
        assert info.iterations <= 10


def test_eval_at_no_points_returns_empty():
    P = WL.poisson1d(levels=(2, 4), features=8, n_interior=40)
    with E.Solver.from_problem(P) as s:
        s.assemble_problem(P)
        s.solve(max_iter=5, atol=0.0, btol=0.0, check_every=5)
        out = s.eval(np.zeros((0, 1)))
    assert out.shape == (0,)


def test_features_past_the_fused_pass_take_the_general_path():
    """K = 160 on a 1-D problem: the k-th LSQR iterate (no preconditioner,
    FP64 panels) equals SciPy's on the oracle's M for k = 1, 2, 3."""
    P = WL.poisson1d(levels=(2, 3), features=160, n_interior=300, lam=100.0)
    ref = OS.assemble(P, fmt="dense")
    for k in (1, 2, 3):
        a_ref = spla.lsqr(ref["M"], ref["h"], atol=0, btol=0, conlim=0, iter_lim=k)[0]
        with E.Solver.from_problem(P, precision=E.FP64) as s:
            s.assemble_problem(P)
            info = s.solve(preconditioner=E.PREC_NONE, max_iter=k, atol=0.0, btol=0.0,
                           check_every=1)
            a = s.coeffs()
        assert info.iterations == k
        assert np.linalg.norm(a - a_ref) <= 1e-10 * np.linalg.norm(a_ref)
    with E.Solver.from_problem(P, precision=E.FP64) as s:
        s.assemble_problem(P)
        with pytest.raises(E.ElmfbError) as ei:
            s.solve(max_iter=5, atol=0.0, btol=0.0, check_every=5)
        assert ei.value.code == E.ERR_UNSUPPORTED


def test_empty_batch_is_a_no_op():
    res, uh, co = E.batch_solve([], precision=E.FP32, n_workers=4)
    assert len(res) == 0 and uh == [] and co == []
