"""PCG on the tensor-core Gram normal equations, with refinement (not in the paper).

The solve claims to return a with (G_bf16 + mu I) a ~= g, g = M^T h, G_bf16
the BF16 tensor-core Gram and mu the Tikhonov shift.  The check uses the
oracle's own matrix: G_bf = bf16(M)^T bf16(M) (M rounded by torch) and
g = M^T h, both in FP64, and measures the relative residual of the GPU
solution in that system.  The GPU Gram differs from G_bf by rounding flips
(<= 2^-9 |M|^T|M|, tests/test_gpu_gram.py), which bounds the attainable
residual at that level times ||a|| |G| / ||g||.
"""
import numpy as np
import pytest

import paper_2409_01949_gb300 as E
import workloads as WL
from oracle import system as OS

pytestmark = pytest.mark.gpu


def _bf16(A):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(A.astype(np.float32)).bfloat16().double().numpy()


def test_pcg_solves_its_normal_equations():
    P = WL.poisson2d(levels=(1, 2), features=16, n_side=24, n_boundary_side=24,
                     modes=[(1.0, 1, 1)])
    ref = OS.assemble(P, fmt="dense")
    M, h = ref["M"], ref["h"]
    Mb = _bf16(M)
    Gb = Mb.T @ Mb
    g = M.T @ h
    frac = 1.0        # well-conditioned system: the check then resolves the BF16 level
    mu = frac * np.trace(Gb) / Gb.shape[0]
    with E.Solver.from_problem(P, precision=E.MIXED) as s:
        s.assemble_problem(P)
        info = s.solve(method=E.SOLVE_PCG, max_iter=200, refine=1, gram_shift=frac, shift=1e-10)
        a = s.coeffs()
    res = np.linalg.norm((Gb + mu * np.eye(len(g))) @ a - g) / np.linalg.norm(g)
    # attainable: Gram rounding flips, 2^-9 |M|^T|M| relative
    floor = 2.0 ** -9 * np.linalg.norm(np.abs(M).T @ np.abs(M) @ np.abs(a)) / np.linalg.norm(g)
    print(f"PCG residual {res:.2e} (rounding floor {floor:.2e}), {info.iterations} its")
    assert res <= max(4 * floor, 1e-6)


def test_refinement_reduces_least_squares_residual():
    P = WL.poisson2d(levels=(1, 2, 4), features=32, n_side=40, n_boundary_side=40)
    ref = OS.assemble(P, fmt="dense")
    M, h = ref["M"], ref["h"]
    res = []
    for refine in (1, 4):
        with E.Solver.from_problem(P, precision=E.MIXED) as s:
            s.assemble_problem(P)
            info = s.solve(method=E.SOLVE_PCG, max_iter=30, refine=refine, gram_shift=1e-4,
                           shift=1e-10)
            a = s.coeffs()
            err = s.error_norms(s.eval(P.test_points), P.exact(P.test_points))["rel_l2"]
        r = float(np.linalg.norm(M @ a - h))
        assert info.residual_norm == pytest.approx(r, rel=1e-4)
        res.append((r, err))
    with E.Solver.from_problem(P, precision=E.MIXED) as s:
        s.assemble_problem(P)
        s.solve(max_iter=120, atol=0, btol=0, shift=1e-10)
        lsqr_err = s.error_norms(s.eval(P.test_points), P.exact(P.test_points))["rel_l2"]
    print(f"PCG+refinement (residual, rel L2): 1 step {res[0]}, 4 steps {res[1]}; "
          f"LSQR 120 its rel L2 {lsqr_err:.2e}")
    assert res[1][0] < res[0][0]


def test_pcg_needs_mixed_precision():
    P = WL.poisson1d(levels=(2,), features=8, n_interior=20)
    with E.Solver.from_problem(P, precision=E.FP64) as s:
        s.assemble_problem(P)
        with pytest.raises(E.ElmfbError) as ei:
            s.solve(method=E.SOLVE_PCG)
        assert ei.value.code == E.ERR_UNSUPPORTED
