"""The seeded input generators (workloads/) against the equations they pose.

* Every row set's right-hand side equals its own operator
  Op[u] = c0 u + sum_i c1_i d_i u + sum_i c2_i d_ii u applied to the problem's
  closed-form solution, by central differences, for each workload family
  (interior PDE rows and every boundary or initial-condition set).
* The generators are deterministic in their seed and differ across seeds.
* The named configurations have the sizes of the hot-path table (rows,
  columns), and the batched draw has 512 instances of the stated ranges.
"""
import numpy as np
import pytest

import workloads as WL


def _op_by_differences(rs, u, X, h):
    """Op[u](X) by central differences, and the size of its largest term."""
    dim = X.shape[1]
    u0 = u(X)
    val = rs.c0 * u0
    scale = np.abs(rs.c0 * u0)
    for i in range(dim):
        e = np.zeros(dim)
        e[i] = h
        up, um = u(X + e), u(X - e)
        d1 = (up - um) / (2 * h)
        d2 = (up - 2 * u0 + um) / (h * h)
        val = val + rs.c1[i] * d1 + rs.c2[i] * d2
        scale = scale + np.abs(rs.c1[i] * d1) + np.abs(rs.c2[i] * d2)
    return val, scale


def _sample(rs, n, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(rs.points.shape[0], min(n, rs.points.shape[0]), replace=False)
    return rs.points[idx], rs.rhs[idx]


PROBLEMS = {
    "poisson1d": lambda: WL.poisson1d(n_interior=400),
    "poisson2d": lambda: WL.poisson2d(n_side=40, n_boundary_side=40),
    "poisson2d_random_modes": lambda: WL.config_poisson2d_large(n_side=64),
    "dho": lambda: WL.dho(n_interior=500),
    "dho_paper_baseline": WL.dho_paper_baseline,
    "laplace_multiscale": lambda: WL.laplace_multiscale(n_grid=20),
    "helmholtz_lshape": lambda: WL.helmholtz_lshape(n_grid=20, n_long=10, n_short=5),
    "batch_instance": lambda: WL.batch_instance(WL.batch_specs(8, 0)[3], 3, 0),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_right_hand_sides_are_the_operator_of_the_exact_solution(name):
    P = PROBLEMS[name]()
    for b, rs in enumerate([P.interior] + list(P.boundary)):
        X, rhs = _sample(rs, 40, b)
        fd, scale = _op_by_differences(rs, P.exact, X, 1e-5)
        tol = 2e-5 * max(scale.max(), np.abs(rhs).max(), 1.0)
        assert np.abs(fd - rhs).max() <= tol, (name, b)


def test_generators_are_deterministic_in_the_seed():
    a = WL.config_poisson2d_large(seed=0, n_side=32)
    b = WL.config_poisson2d_large(seed=0, n_side=32)
    c = WL.config_poisson2d_large(seed=1, n_side=32)
    assert np.array_equal(a.interior.rhs, b.interior.rhs)
    assert not np.array_equal(a.interior.rhs, c.interior.rhs)
    s0, s0b, s1 = WL.batch_specs(512, 0), WL.batch_specs(512, 0), WL.batch_specs(512, 1)
    assert s0 == s0b and s0 != s1


def test_named_configurations_have_the_table_sizes():
    P1 = WL.config_poisson1d()
    assert (P1.n_rows, P1.n_columns) == (2002, 16 * 64)
    P2 = WL.config_poisson2d_ml()
    assert (P2.n_rows, P2.n_columns) == (160000 + 1600, 341 * 128)
    P3 = WL.config_dho_ml()
    assert (P3.n_rows, P3.n_columns) == (20000 + 2, 127 * 96)
    P5 = WL.config_poisson2d_large()
    assert (P5.n_rows, P5.n_columns) == (2048 * 2048 + 8192, 5461 * 64)


def test_batched_draw_ranges():
    specs = WL.batch_specs(512, 0)
    assert len(specs) == 512
    assert all(2 <= s.n_sub <= 32 and s.features in (32, 64, 128) for s in specs)
    assert {s.features for s in specs} == {32, 64, 128}
    assert sum(s.n_sub ** 2 * s.features for s in specs) == 14934304
