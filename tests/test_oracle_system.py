"""Pins of the oracle's least-squares system (§3 definitions of f, g, N, B)."""
import dataclasses
import math

import numpy as np
import pytest

import workloads as WL
from oracle import decomposition as D
from oracle import evaluate as E
from oracle import features as F
from oracle import system as S
from oracle import windows as Wn


def _small_2d():
    return WL.poisson2d(levels=(1, 2, 3), features=5, n_side=9, n_boundary_side=4,
                        delta=2.0, seed=11)


def _small_dho():
    return WL.dho(levels=(1, 3), features=6, n_interior=25, omega0=9.0, zeta=0.3, seed=5)


def _g(problem, X, lev_index, j, k, params):
    """x -> w_j(x) phi_jk(x) evaluated from the window and feature definitions."""
    d = problem.dim
    lev = D.build_levels(d, problem.lo, problem.hi, problem.levels, problem.delta,
                         problem.features, problem.placement)[lev_index]
    w = Wn.level_windows(X, lev, d)["om"][:, j]
    ji = D.subdomain_multi_index(lev, d, j)
    mu = np.array([lev.mu[i][ji[i]] for i in range(d)])
    sig = np.array(lev.sigma)
    q = lev.col_offset + j * problem.features + k
    W, b = params
    phi = F.features((X - mu) / sig, W[q:q + 1], b[q:q + 1], sig)[0][:, 0]
    return w * phi, q


@pytest.mark.parametrize("make", [_small_2d, _small_dho])
def test_entries_equal_operator_applied_by_finite_differences(make):
    P = make()
    out = S.assemble(P, fmt="dense", with_bound=True)
    M, bound = out["M"], out["bound"]
    R = S.stack_rows(P)
    params = S.parameters(P)
    L = len(P.levels)
    d = P.dim
    rng = np.random.default_rng(0)
    checked = 0
    for lev_index, n in enumerate(P.levels):
        for j in rng.choice(n ** d, size=min(3, n ** d), replace=False):
            k = int(rng.integers(P.features))
            g0, q = _g(P, R.X, lev_index, int(j), k, params)
            val = R.c0 * g0
            for i in range(d):
                sig_min = min(D.build_levels(d, P.lo, P.hi, P.levels, P.delta, P.features)[lev_index].sigma)
                e = 2e-4 * sig_min
                Xp = R.X.copy(); Xp[:, i] += e
                Xm = R.X.copy(); Xm[:, i] -= e
                gp, _ = _g(P, Xp, lev_index, int(j), k, params)
                gm, _ = _g(P, Xm, lev_index, int(j), k, params)
                val = val + R.c1[:, i] * (gp - gm) / (2 * e) + R.c2[:, i] * (gp - 2 * g0 + gm) / e ** 2
            ref = R.scale * val / L
            blk = slice(q - k, q - k + P.features)
            # the finite-difference truncation error is absolute, set by the block's scale
            tol = 2e-5 * np.maximum(bound[:, blk].max(axis=1), 1e-3 * bound[:, blk].max())
            inside = np.abs(M[:, q]) > 0
            assert np.all(np.abs(M[inside, q] - ref[inside]) <= tol[inside])
            checked += int(inside.sum())
    assert checked > 50


def test_single_subdomain_reduces_to_plain_elm_column():
    """J = 1 with a support covering the domain: w = 1, so N_{n,q} = N[phi_q](x_n) / sqrt(N_I)."""
    P = WL.poisson1d(levels=(1,), features=7, n_interior=50, delta=2.0)
    M = S.assemble(P, fmt="dense")["M"]
    W, b = S.parameters(P)
    x = P.interior.points[:, 0]
    sig = 1.0  # delta * Delta / 2 with Delta = 1
    s = np.outer((x - 0.5) / sig, W[:, 0]) + b
    phi = np.tanh(s)
    minus_phi_xx = 2 * phi * (1 - phi ** 2) * (W[:, 0] / sig) ** 2
    assert np.allclose(M[:50], minus_phi_xx / math.sqrt(50), rtol=1e-12, atol=1e-14)
    lam = P.boundary[0].weight
    assert np.allclose(M[50:], math.sqrt(lam / 2) * np.tanh(np.outer(([0, 1] - 0.5 * np.ones(2)) / sig, W[:, 0]) + b),
                       rtol=1e-12)


def test_zero_weights_give_constant_feature_times_window_operator():
    """w = 0: phi = tanh(b) is constant, so Op[w phi] = tanh(b) Op[w]."""
    P = _small_2d()
    W, b = S.parameters(P)
    params = (np.zeros_like(W), b)
    M = S.assemble(P, fmt="dense", params=params)["M"]
    R = S.stack_rows(P)
    L = len(P.levels)
    levels = D.build_levels(2, P.lo, P.hi, P.levels, P.delta, P.features)
    for lev in levels:
        win = Wn.level_windows(R.X, lev, 2)
        for j in range(lev.n_sub):
            opw = R.c0 * win["om"][:, j] + (R.c1 * win["dom"][:, j, :]).sum(1) + \
                (R.c2 * win["ddom"][:, j, :]).sum(1)
            q0 = lev.col_offset + j * P.features
            ref = np.outer(R.scale * opw / L, np.tanh(b[q0:q0 + P.features]))
            assert np.allclose(M[:, q0:q0 + P.features], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("make", [_small_2d, _small_dho])
def test_residual_norm_equals_physics_loss(make):
    """||M a - h||^2 = L(a) of Eq. multilevel_loss, with the operators applied to u_hat by finite differences."""
    P = make()
    out = S.assemble(P, fmt="dense")
    M, h = out["M"], out["h"]
    rng = np.random.default_rng(3)
    a = rng.standard_normal(P.n_columns)
    lhs = float(np.sum((M @ a - h) ** 2))
    d = P.dim
    e = 1e-4 * min(1.0 / max(P.levels), 1.0)

    def op_uhat(rs):
        X = rs.points
        u0 = E.u_hat(P, a, X)
        v = rs.c0 * u0
        for i in range(d):
            Xp = X.copy(); Xp[:, i] += e
            Xm = X.copy(); Xm[:, i] -= e
            up = E.u_hat(P, a, Xp)
            um = E.u_hat(P, a, Xm)
            v = v + rs.c1[i] * (up - um) / (2 * e) + rs.c2[i] * (up - 2 * u0 + um) / e ** 2
        return v

    NI = P.interior.points.shape[0]
    loss = float(np.sum((op_uhat(P.interior) - P.interior.rhs) ** 2)) / NI
    for bs in P.boundary:
        NB = bs.points.shape[0]
        loss += bs.weight / NB * float(np.sum((op_uhat(bs) - bs.rhs) ** 2))
    assert lhs == pytest.approx(loss, rel=2e-5)


def test_rhs_scaling_and_row_order():
    P = _small_dho()
    h = S.rhs_vector(P)
    NI = P.interior.points.shape[0]
    assert np.allclose(h[:NI], P.interior.rhs / math.sqrt(NI))
    assert h[NI] == pytest.approx(math.sqrt(P.boundary[0].weight) * 1.0)
    assert h[NI + 1] == 0.0


def test_nonzero_count_closed_form_poisson1d():
    """2000 midpoints, 16 cell-centred subdomains, delta = 2, K = 64.

    A point strictly between two neighbouring centres lies in 2 open supports,
    a point on a centre or outside [mu_0, mu_15] in 1: 62+1+1860*2+14+1+62 =
    3860 interior row-subdomain pairs, plus 1 for each of x = 0 and x = 1:
    3862 * 64 = 247168 entries.
    """
    P = WL.config_poisson1d()
    M = S.assemble(P, fmt="csr")["M"]
    assert M.nnz == 247168
    assert M.shape == (2002, 1024)


def test_lshape_discards_the_subdomains_of_the_cut_out_square():
    """§4.4 baseline: a 16 x 16 grid minus the 8 x 8 subdomains outside the
    L-shaped domain leaves 192 subdomains (3072 columns at K = 16); a 32 x 32
    level keeps 1024 - 256 = 768, the single level-1 subdomain (centre on the
    corner of the cut) is kept."""
    P = WL.helmholtz_lshape()
    assert D.n_columns(P) == 192 * 16
    assert D.n_columns(WL.helmholtz_lshape(placement="endpoint")) == 192 * 16
    P3 = WL.helmholtz_lshape(levels=(1, 16, 32))
    levels = D.build_levels(2, P3.lo, P3.hi, P3.levels, P3.delta, P3.features, P3.placement,
                            P3.holes)
    assert [int(l.keep.sum()) for l in levels] == [1, 192, 768]
    assert D.n_columns(P3) == (1 + 192 + 768) * 16


def test_lshape_windows_partition_unity_over_kept_subdomains():
    """At every interior and boundary point of the L-shape the kept windows of
    each level still sum to 1 and their derivatives to 0 (the discarded ones
    take no part in the normalisation)."""
    P = WL.helmholtz_lshape(levels=(1, 16, 32))
    X = np.concatenate([P.interior.points, P.boundary[0].points])
    levels = D.build_levels(2, P.lo, P.hi, P.levels, P.delta, P.features, P.placement, P.holes)
    for lev in levels:
        w = Wn.level_windows(X, lev, 2)
        assert np.all(w["om"][:, ~lev.keep] == 0.0)
        assert np.allclose(w["om"].sum(axis=1), 1.0, atol=1e-13)
        assert np.allclose(w["dom"].sum(axis=1), 0.0, atol=1e-9 * np.abs(w["dom"]).max() + 1e-12)
        assert np.allclose(w["ddom"].sum(axis=1), 0.0,
                           atol=1e-9 * np.abs(w["ddom"]).max() + 1e-12)


def test_helmholtz_source_matches_operator_by_finite_differences():
    """The workload's f (Eq. helmholtz_f) equals Laplace u + k^2 u of its u (Eq.
    helmholtz_exact), by central differences at scattered L-shape points."""
    P = WL.helmholtz_lshape()
    rng = np.random.default_rng(3)
    X = P.interior.points[rng.choice(P.interior.points.shape[0], 40, replace=False)]
    h = 1e-4
    u = P.exact
    lap = sum((u(X + h * e) - 2 * u(X) + u(X - h * e)) / h ** 2
              for e in (np.array([1.0, 0.0]), np.array([0.0, 1.0])))
    k2 = P.interior.c0
    fd = lap + k2 * u(X)
    f = P.interior.rhs[[int(np.nonzero((P.interior.points == x).all(axis=1))[0][0]) for x in X]]
    assert np.allclose(fd, f, rtol=0, atol=2e-5 * np.abs(f).max())


def test_lshape_assembly_columns_of_a_kept_subdomain_use_its_full_grid_parameters():
    """Discarding renumbers columns but keeps each subdomain's parameter draw:
    the assembled column block of a kept subdomain equals the same block of
    the undiscarded problem at the rows that subdomain covers away from the
    cut (where no discarded window entered the normalisation)."""
    P = WL.helmholtz_lshape(n_grid=24, n_long=8, n_short=4)
    Pf = dataclasses.replace(P, holes=())
    rows = np.nonzero((P.interior.points[:, 0] < 0.3) & (P.interior.points[:, 1] < 0.3))[0]
    A = S.assemble(P, rows=rows, fmt="dense")["M"]
    B = S.assemble(Pf, rows=rows, fmt="dense")["M"]
    levels = D.build_levels(2, P.lo, P.hi, P.levels, P.delta, P.features, P.placement, P.holes)
    lev = levels[0]
    K = P.features
    for j in (0, 1, 16, 17):           # subdomains near the (0, 0) corner, all kept
        assert lev.keep[j]
        c = int(lev.col_first[j])
        assert np.array_equal(A[:, c:c + K], B[:, j * K:(j + 1) * K])


def test_ansatz_vanishes_on_the_boundary_and_matches_finite_differences():
    """§4.3: A(x) = prod_i tanh(w (x_i - lo_i)) tanh(w (hi_i - x_i)) is zero on
    the box boundary; dA and ddA equal central differences of A."""
    from oracle import ansatz as AZ
    rng = np.random.default_rng(4)
    Xb = np.array([[0.0, 0.3], [1.0, 0.6], [0.2, 0.0], [0.9, 1.0]])
    assert np.all(AZ.ansatz(Xb, (0, 0), (1, 1), 16.0)[0] == 0.0)
    X = rng.uniform(0.05, 0.95, size=(30, 2))
    A, dA, ddA = AZ.ansatz(X, (0, 0), (1, 1), 6.0)
    h = 1e-5
    for i in range(2):
        e = np.zeros(2); e[i] = h
        Ap = AZ.ansatz(X + e, (0, 0), (1, 1), 6.0)[0]
        Am = AZ.ansatz(X - e, (0, 0), (1, 1), 6.0)[0]
        assert np.allclose(dA[:, i], (Ap - Am) / (2 * h), rtol=1e-7, atol=1e-8)
        assert np.allclose(ddA[:, i], (Ap - 2 * A + Am) / h ** 2, rtol=1e-4, atol=1e-3)


def test_ansatz_entries_equal_operator_applied_by_finite_differences():
    """With the ansatz the entry of column q at row x is -Laplace[A w_j phi_jk](x)
    / (sqrt(N_I) L): central differences of x -> A(x) w_j(x) phi_jk(x)."""
    from oracle import ansatz as AZ
    P = WL.laplace_multiscale(omegas=(2, 3), levels=(1, 3), features=4, n_grid=12, delta=2.0)
    out = S.assemble(P, fmt="dense", with_bound=True)
    M, bound = out["M"], out["bound"]
    R = S.stack_rows(P)
    params = S.parameters(P)
    L = len(P.levels)
    checked = 0
    for lev_index, n in enumerate(P.levels):
        for j in range(n * n):
            k = j % P.features

            def g(X):
                v, q = _g(P, X, lev_index, j, k, params)
                return AZ.ansatz(X, P.lo, P.hi, P.ansatz_omega)[0] * v, q
            g0, q = g(R.X)
            e = 2e-4 * min(D.build_levels(2, P.lo, P.hi, P.levels, P.delta,
                                          P.features)[lev_index].sigma)
            lap = 0.0
            for i in range(2):
                Xp = R.X.copy(); Xp[:, i] += e
                Xm = R.X.copy(); Xm[:, i] -= e
                lap = lap + (g(Xp)[0] - 2 * g0 + g(Xm)[0]) / e ** 2
            ref = R.scale * (-lap) / L
            blk = slice(q - k, q - k + P.features)
            tol = 2e-5 * np.maximum(bound[:, blk].max(axis=1), 1e-3 * bound[:, blk].max())
            inside = np.abs(M[:, q]) > 0
            assert np.all(np.abs(M[inside, q] - ref[inside]) <= tol[inside])
            checked += int(inside.sum())
    assert checked > 50


def test_ansatz_model_is_zero_on_the_boundary():
    P = WL.laplace_multiscale(omegas=(2, 3), levels=(1, 3), features=4, n_grid=12)
    a = np.random.default_rng(2).standard_normal(P.n_columns)
    Xb = WL.square_boundary_midpoints(7)
    assert np.all(E.u_hat(P, a, Xb) == 0.0)
    assert np.any(E.u_hat(P, a, P.interior.points) != 0.0)
