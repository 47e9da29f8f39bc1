"""Precision requirements of the stored system, established with the oracle.

The condition numbers of M reach 1e17-1e20 (the paper's tables report up to
~3e20), and the accurate solutions use singular directions far below FP32
resolution.  Rounding M's entries to FP32 therefore bounds the attainable
error, independently of the solver: the exact least-squares solution of the
FP32-rounded matrix is worse than the FP64 paper-protocol LSQR result on the
damped oscillator.  This is why the oscillator workload keeps FP64 panels.
"""
import numpy as np

import workloads as WL
from oracle import evaluate as E
from oracle import lstsq as LS
from oracle import system as S


def _err(P, M, h):
    a, _ = LS.lstsq_qr(M, h)
    return E.rel_l2(E.u_hat(P, a, P.test_points), P.exact(P.test_points))


def test_fp32_rounded_matrix_limits_the_oscillator():
    P = WL.dho(levels=(1, 2, 4, 8), features=24, n_interior=1000)
    out = S.assemble(P, fmt="dense")
    M, h = out["M"], out["h"]
    e64 = _err(P, M, h)
    e32 = _err(P, M.astype(np.float32).astype(np.float64), h)
    a, _ = LS.lstsq_lsqr(M, h, iter_lim=15000)
    e_paper = E.rel_l2(E.u_hat(P, a, P.test_points), P.exact(P.test_points))
    assert e64 < 1e-4
    assert e32 > 100 * e64
    assert e32 > e_paper
