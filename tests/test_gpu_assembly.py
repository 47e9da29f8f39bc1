"""GPU parity of create (parameters) and assembly (M, h) against the FP64 oracle.

Tolerance on entries (paper §3 entries; precision reading): |M_gpu - M_oracle|
<= tol * max(T, 1e-3 S), with T the largest magnitude sum of product-rule and
quotient-rule terms over the K features of the same row and subdomain block
(the oracle's ``bound``), S the largest T of that subdomain block over all
rows, tol = 1e-12 for FP64 and DF32 (FP32 pair) panels and 1e-6 for FP32
panels.  The 1e-3 S floor
covers points within rounding distance of a support edge, where the window and
its derivatives vanish and an entry's relative value is not determined by the
FP64 coordinates.
"""
import numpy as np
import pytest

import paper_2409_01949_gb300 as E
import workloads as WL
from oracle import decomposition as OD
from oracle import rng as OR
from oracle import system as OS

pytestmark = pytest.mark.gpu

TOL = {E.FP64: 1e-12, E.FP32: 1e-6, E.MIXED: 1e-6, E.DF32: 1e-12}

SMALL = {
    "poisson1d_full": (WL.config_poisson1d, [E.FP64, E.FP32, E.DF32]),
    "dho_L1-8_K24": (lambda: WL.dho(levels=(1, 2, 4, 8), features=24, n_interior=1000),
                     [E.FP64, E.FP32, E.DF32]),
    "poisson2d_L1-4_K64": (lambda: WL.poisson2d(levels=(1, 2, 4), features=64, n_side=60,
                                                n_boundary_side=60),
                           [E.FP64, E.FP32, E.MIXED, E.DF32]),
    "dho_paper_K12_delta2.9_endpoint": (WL.dho_paper_baseline, [E.FP64]),
    "poisson2d_delta2.9_K40": (lambda: WL.poisson2d(levels=(3, 5), features=40, n_side=50,
                                                    n_boundary_side=50, delta=2.9), [E.FP32]),
    "poisson2d_ragged_K33": (lambda: WL.poisson2d(levels=(1, 3, 7), features=33, n_side=37,
                                                  n_boundary_side=11),
                            [E.FP64, E.FP32, E.DF32]),
    # §4.4: the L-shaped domain, subdomains of the cut-out square discarded
    "helmholtz_L_w8_J16_K16": (WL.helmholtz_lshape, [E.FP64, E.FP32, E.DF32]),
    "helmholtz_L_J1-8-16_K12_endpoint": (
        lambda: WL.helmholtz_lshape(levels=(1, 8, 16), features=12, n_grid=40, n_long=40,
                                    n_short=20, placement="endpoint"), [E.FP64, E.DF32]),
    # the largest feature counts: K = 256 (the library's maximum), K = 160 (past
    # the fused pass's 128, ragged against 32-lane slices)
    "poisson1d_Kmax256": (lambda: WL.poisson1d(levels=(2, 4), features=256, n_interior=90),
                          [E.FP64, E.FP32, E.DF32]),
    "poisson2d_K160": (lambda: WL.poisson2d(levels=(2,), features=160, n_side=26,
                                            n_boundary_side=9), [E.FP64, E.FP32]),
    # §4.3: the hard-constraint ansatz, no boundary rows
    "laplace_n4_J16_K16": (WL.laplace_multiscale, [E.FP64, E.FP32, E.DF32]),
    "laplace_n2_J1-4-8_K20_ansatz": (
        lambda: WL.laplace_multiscale(omegas=(3, 5), levels=(1, 4, 8), features=20, n_grid=30,
                                      delta=2.0), [E.FP64, E.FP32]),
}


def _scale(bound, K):
    T = OS.block_max(bound, K)
    S = T.max(axis=0, keepdims=True)
    return np.maximum(T, 1e-3 * S)


def _compare(P, prec, rows=None):
    with E.Solver.from_problem(P, precision=prec) as s:
        s.assemble_problem(P)
        sz = s.sizes()
        rows = np.arange(P.n_rows) if rows is None else np.asarray(rows)
        Mg, hg = s.get_rows(rows)
        ref = OS.assemble(P, rows=rows, fmt="dense", with_bound=True)
        scale = _scale(ref["bound"], P.features)
        err = np.abs(Mg - ref["M"])
        ratio = float((err / np.maximum(scale, 1e-300)).max())
        assert np.all(err <= TOL[prec] * scale), f"max err/scale = {ratio:.3e}"
        assert np.allclose(hg, ref["h"], rtol=1e-15, atol=0)
        return sz, ratio


@pytest.mark.parametrize("name", list(SMALL))
def test_assembly_all_rows(name):
    make, precs = SMALL[name]
    P = make()
    for prec in precs:
        sz, ratio = _compare(P, prec)
        assert sz.n_rows == P.n_rows and sz.n_columns == OD.n_columns(P)


def test_stored_entry_count_matches_closed_form():
    """1D Poisson, 16 cell-centred subdomains, delta = 2, 2000 midpoints, K = 64.

    The oracle's nonzeros are 3862 row-subdomain pairs (247168 entries).  The
    panels also store, as exact zeros, the 15 centre points mu_0..mu_14 that
    lie on the left edge of the open support of their right neighbour (they
    share that neighbour's cell): 3877 * 64 = 248128 stored entries.
    """
    P = WL.config_poisson1d()
    with E.Solver.from_problem(P, precision=E.FP64) as s:
        s.assemble_problem(P)
        assert s.sizes().nnz == 248128


def test_parameters_bitwise_equal_to_oracle_stream():
    P = WL.poisson2d(levels=(1, 2, 4), features=16, n_side=8)
    with E.Solver.from_problem(P) as s:
        W, b = s.params()
    Wo, bo = OR.draw_parameters(P.seed, P.n_columns, 2, P.weight_scale)
    assert np.array_equal(W, Wo) and np.array_equal(b, bo)


def test_discarded_subdomains_keep_their_parameter_draws():
    """With holes the kept columns carry the draws of their full-grid columns
    (the oracle's stream restricted to the kept subdomains)."""
    P = WL.helmholtz_lshape(levels=(1, 4, 8), features=8)
    levels = OD.build_levels(2, P.lo, P.hi, P.levels, P.delta, P.features, P.placement, P.holes)
    full = np.concatenate([lev.param_offset + np.arange(lev.n_sub * P.features)
                           .reshape(lev.n_sub, P.features)[lev.keep].ravel() for lev in levels])
    with E.Solver.from_problem(P) as s:
        W, b = s.params()
        assert s.sizes().n_subdomains == sum(int(l.keep.sum()) for l in levels)
    Wo, bo = OR.draw_parameters(P.seed, P.n_columns_full, 2, P.weight_scale)
    assert np.array_equal(W, Wo[full]) and np.array_equal(b, bo[full])


@pytest.mark.parametrize("maker,prec", [(WL.config_poisson2d_ml, E.FP32),
                                        (WL.config_dho_ml, E.FP32),
                                        (WL.config_poisson2d_large, E.FP32)])
def test_assembly_full_size_sampled_rows(maker, prec):
    """Full workload sizes, as assembled for the benchmark; rows sampled for the oracle."""
    P = maker()
    rng = np.random.default_rng(7)
    NI = P.interior.points.shape[0]
    rows = np.unique(np.concatenate([rng.choice(NI, 200, replace=False), [0, NI - 1],
                                     NI + rng.choice(P.n_rows - NI, min(32, P.n_rows - NI),
                                                     replace=False)]))
    _compare(P, prec, rows)


def test_out_of_box_point_rejected():
    P = WL.poisson1d(levels=(4,), features=8, n_interior=20)
    pts = P.interior.points.copy()
    pts[3, 0] = 1.5
    with E.Solver.from_problem(P) as s:
        with pytest.raises(E.ElmfbError) as ei:
            s.assemble([dict(points=pts, rhs=P.interior.rhs, c2=(-1.0,))])
        assert ei.value.code == E.ERR_INVALID_ARG


def test_invalid_config_rejected():
    with pytest.raises(E.ElmfbError) as ei:
        E.Solver(1, (0.0,), (1.0,), (4,), delta=1.0, features=8)
    assert ei.value.code == E.ERR_INVALID_ARG


def test_empty_boundary_set_and_boundary_points():
    """A boundary set with zero points is allowed; points on the box edge are inside."""
    P = WL.poisson1d(levels=(2, 4), features=8, n_interior=30)
    sets = [dict(points=P.interior.points, rhs=P.interior.rhs, c2=(-1.0,)),
            dict(points=np.zeros((0, 1)), rhs=np.zeros(0), c0=1.0, weight=1.0, n=0),
            dict(points=np.array([[0.0], [1.0]]), rhs=np.zeros(2), c0=1.0, weight=4.0)]
    with E.Solver.from_problem(P) as s:
        s.assemble(sets)
        assert s.sizes().n_rows == 32
