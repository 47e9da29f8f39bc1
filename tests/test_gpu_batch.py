"""Batched solves of uneven independent instances (not in the paper).

* elmfb_batch_solve (several host workers and streams) returns, for every
  instance, bitwise the coefficients and u_hat of a one-by-one solve;
* each instance's relative L2 error is within 1.01x the oracle's
  paper-protocol error (SciPy LSQR, 15000 iterations) on small instances.
"""
import numpy as np
import pytest

import paper_2409_01949_gb300 as E
import workloads as WL
from oracle import evaluate as OE
from oracle import lstsq as OL
from oracle import system as OS

pytestmark = pytest.mark.gpu


def _instances(n, cap_side=96, cap_sub=6, seed=0):
    specs = WL.batch_specs(n, seed)
    out = []
    for i, sp in enumerate(specs):
        sp = WL.BatchSpec(n_sub=min(sp.n_sub, cap_sub), features=sp.features,
                          n_side=min(sp.n_side, cap_side), k=sp.k)
        out.append(WL.batch_instance(sp, i, seed))
    return out


def test_batch_equals_one_by_one():
    probs = _instances(10)
    opts = E.default_solve_opts(max_iter=150, atol=0.0, btol=0.0, shift=1e-10)
    res, uh, co = E.batch_solve(probs, precision=E.FP32, n_workers=4, opts=opts, coeffs=True)
    assert all(r.status == E.OK for r in res)
    for P, u_b, a_b in zip(probs, uh, co):
        with E.Solver.from_problem(P, precision=E.FP32) as s:
            s.assemble_problem(P)
            s.solve(opts)
            a = s.coeffs()
            u = s.eval(P.test_points)
        assert np.array_equal(a, a_b)
        assert np.array_equal(u, u_b)


def test_batch_errors_match_paper_protocol_on_small_instances():
    probs = [P for P in _instances(24, cap_side=64, cap_sub=3) if P.features <= 64][:3]
    opts = E.default_solve_opts(max_iter=2000, atol=1e-12, btol=1e-12, shift=1e-10)
    res, uh, _ = E.batch_solve(probs, precision=E.FP64, n_workers=3, opts=opts)
    for P, r in zip(probs, res):
        out = OS.assemble(P, fmt="dense")
        a, _ = OL.lstsq_lsqr(out["M"], out["h"], iter_lim=15000)
        e_or = OE.rel_l2(OE.u_hat(P, a, P.test_points), P.exact(P.test_points))
        print(f"{P.name}: n_sub {P.levels[0]}^2 K {P.features} rows {P.n_rows}: "
              f"batch rel L2 {r.rel_l2:.3e} ({r.iterations} its), oracle LSQR-15000 {e_or:.3e}")
        assert r.rel_l2 <= 1.01 * e_or
