"""Seeded synthetic inputs for the multilevel ELM-FBPINN solver.

This module is the only code shared by the CUDA path (through ``bench.py`` and
the tests) and the FP64 CPU oracle.  It holds problem *data* only: domains,
collocation points, operator coefficients, penalty weights, right-hand sides and
closed-form solutions.  It contains none of the method's arithmetic (no
windows, no features, no scalings, no assembly, no solve): every side computes
those itself.

Problem statement follows the paper's §3 "Problem and model definition":
a linear operator N[u] = f on the interior points and linear boundary operators
B_b[u] = g_b on boundary point sets, each boundary set carrying its own penalty
weight lambda_b (Eq. ``multilevel_loss``).  Operators are restricted to the
constant-coefficient family

    Op[v] = c0 v + sum_i c1[i] d_i v + sum_i c2[i] d_ii v

which covers every PDE and boundary condition of §4 (damped oscillator,
Laplace/Poisson, Helmholtz, Dirichlet and Neumann-type initial conditions).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class RowSet:
    """One block of rows of the least-squares system (§3, Eq. ``multilevel_ls``).

    ``weight`` is None for the interior PDE rows (row scale 1/sqrt(N_I)) and
    lambda_b for a boundary set (row scale sqrt(lambda_b / N_B^(b))).
    """

    points: np.ndarray          # (n, dim) float64, row-major
    c0: float
    c1: Tuple[float, ...]       # length dim
    c2: Tuple[float, ...]       # length dim
    rhs: np.ndarray             # (n,) float64: f or g_b at the points
    weight: Optional[float] = None


@dataclasses.dataclass
class Problem:
    """A complete multilevel ELM-FBPINN instance (data only)."""

    name: str
    dim: int
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    levels: Tuple[int, ...]     # subdomains per dimension at each level, coarse to fine
    delta: float                # width ratio (§4.1 "Domain decomposition")
    features: int               # K, random features per subdomain
    seed: int                   # parameter stream seed
    weight_scale: float         # a: parameters ~ U(-a, a)
    interior: RowSet
    boundary: List[RowSet]
    exact: Callable[[np.ndarray], np.ndarray]
    test_points: np.ndarray     # (m, dim) float64
    placement: str = "cell"     # subdomain centres: "cell" (cell-centred) or "endpoint"
    # boxes ((lo_x, lo_y), (hi_x, hi_y)) cut out of the domain; subdomains whose
    # centre lies inside one are discarded (§4.1, the L-shape of §4.4)
    holes: Tuple = ()
    # > 0: hard-constraint ansatz u~ = A u_hat, A = prod_i tanh(w (x_i - lo_i))
    # tanh(w (hi_i - x_i)) (§4.3); the problem then has no boundary rows
    ansatz_omega: float = 0.0

    @property
    def n_rows(self) -> int:
        return self.interior.points.shape[0] + sum(b.points.shape[0] for b in self.boundary)

    @property
    def n_subdomains_full(self) -> int:
        """Subdomains of the full grids, before any are discarded."""
        return sum(n ** self.dim for n in self.levels)

    @property
    def n_columns_full(self) -> int:
        return self.features * self.n_subdomains_full

    @property
    def n_subdomains(self) -> int:
        if self.holes:
            raise AttributeError("with holes the count depends on the subdomain centres: "
                                 "ask the solver (sizes) or the oracle (decomposition)")
        return self.n_subdomains_full

    @property
    def n_columns(self) -> int:
        return self.features * self.n_subdomains


# ----------------------------------------------------------------------------
# point sets
# ----------------------------------------------------------------------------

def midpoints(n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n cell-centred points (i + 1/2) (hi - lo) / n + lo."""
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def grid2d(xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """Tensor grid, raster order with x fastest: point index = iy * len(xs) + ix."""
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def square_boundary_midpoints(n: int) -> np.ndarray:
    """n midpoints on each side of [0,1]^2 (no corners): bottom, right, top, left."""
    m = midpoints(n)
    z = np.zeros(n)
    o = np.ones(n)
    return np.concatenate([
        np.stack([m, z], 1),
        np.stack([o, m], 1),
        np.stack([m[::-1], o], 1),
        np.stack([z, m[::-1]], 1),
    ])


# ----------------------------------------------------------------------------
# problem families
# ----------------------------------------------------------------------------

def poisson1d(levels=(16,), features=64, n_interior=2000, delta=2.0, seed=0,
              weight_scale=1.0, lam=None, name="poisson1d") -> Problem:
    """-u'' = f on [0,1], u(0) = u(1) = 0, u = sin(2 pi x) + 0.1 sin(50 pi x)."""
    if lam is None:
        lam = (50.0 * math.pi) ** 4

    def u(x):
        x = np.asarray(x)[..., 0]
        return np.sin(2 * math.pi * x) + 0.1 * np.sin(50 * math.pi * x)

    def f(x):
        x = np.asarray(x)[..., 0]
        return (4 * math.pi ** 2) * np.sin(2 * math.pi * x) + \
            0.1 * (50 * math.pi) ** 2 * np.sin(50 * math.pi * x)

    xi = midpoints(n_interior)[:, None]
    xb = np.array([[0.0], [1.0]])
    return Problem(
        name=name, dim=1, lo=(0.0,), hi=(1.0,), levels=tuple(levels), delta=delta,
        features=features, seed=seed, weight_scale=weight_scale,
        interior=RowSet(xi, 0.0, (0.0,), (-1.0,), f(xi)),
        boundary=[RowSet(xb, 1.0, (0.0,), (0.0,), u(xb), weight=lam)],
        exact=u, test_points=np.linspace(0.0, 1.0, 1000)[:, None])


def _sine_modes_2d(modes):
    """u = sum A sin(k pi x) sin(l pi y); returns (u, -Laplace u)."""
    def u(p):
        p = np.asarray(p)
        out = np.zeros(p.shape[:-1])
        for A, k, l in modes:
            out = out + A * np.sin(k * math.pi * p[..., 0]) * np.sin(l * math.pi * p[..., 1])
        return out

    def f(p):
        p = np.asarray(p)
        out = np.zeros(p.shape[:-1])
        for A, k, l in modes:
            out = out + A * (k * k + l * l) * math.pi ** 2 * \
                np.sin(k * math.pi * p[..., 0]) * np.sin(l * math.pi * p[..., 1])
        return out
    return u, f


def poisson2d(levels=(1, 2, 4, 8, 16), features=128, n_side=400, delta=2.0, seed=0,
              weight_scale=1.0, modes=None, lam=None, n_boundary_side=None,
              n_test_side=96, name="poisson2d") -> Problem:
    """-Laplace u = f on [0,1]^2, u = 0 on the boundary.

    Default modes: u = sum_{k=1..4} 2^-k sin(2^k pi x) sin(2^k pi y).
    """
    if modes is None:
        modes = [(2.0 ** -k, 2 ** k, 2 ** k) for k in range(1, 5)]
    if lam is None:
        kmax = max(max(k, l) for _, k, l in modes)
        lam = (kmax * math.pi) ** 4
    if n_boundary_side is None:
        n_boundary_side = n_side
    u, f = _sine_modes_2d(modes)
    xi = grid2d(midpoints(n_side), midpoints(n_side))
    xb = square_boundary_midpoints(n_boundary_side)
    t = np.linspace(0.0, 1.0, n_test_side)
    return Problem(
        name=name, dim=2, lo=(0.0, 0.0), hi=(1.0, 1.0), levels=tuple(levels), delta=delta,
        features=features, seed=seed, weight_scale=weight_scale,
        interior=RowSet(xi, 0.0, (0.0, 0.0), (-1.0, -1.0), f(xi)),
        boundary=[RowSet(xb, 1.0, (0.0, 0.0), (0.0, 0.0), u(xb), weight=lam)],
        exact=u, test_points=grid2d(t, t))


def dho(levels=(1, 2, 4, 8, 16, 32, 64), features=96, n_interior=20000, omega0=80.0,
        zeta=0.2, beta=None, delta=2.0, seed=0, weight_scale=1.0, n_test=1000,
        placement="cell", name="dho") -> Problem:
    """Damped harmonic oscillator (§4.2, Eq. ``harm_oscillator``) with m = 1.

    u'' + 2 beta u' + omega0^2 u = 0 on (0,1], u(0) = 1, u'(0) = 0, with
    beta = zeta * omega0 unless given.  Penalties lambda_u0 = omega0^4 and
    lambda_v0 = omega0^2 (§4.2 "Physics-informed objective").  Collocation
    t_i = i / N, i = 1..N.
    """
    if beta is None:
        beta = zeta * omega0
    w = math.sqrt(omega0 ** 2 - beta ** 2)

    def u(t):
        t = np.asarray(t)[..., 0]
        return np.exp(-beta * t) * (np.cos(w * t) + (beta / w) * np.sin(w * t))

    ti = (np.arange(1, n_interior + 1, dtype=np.float64) / n_interior)[:, None]
    t0 = np.zeros((1, 1))
    return Problem(
        name=name, dim=1, lo=(0.0,), hi=(1.0,), levels=tuple(levels), delta=delta,
        features=features, seed=seed, weight_scale=weight_scale,
        interior=RowSet(ti, omega0 ** 2, (2.0 * beta,), (1.0,), np.zeros(n_interior)),
        boundary=[RowSet(t0, 1.0, (0.0,), (0.0,), np.ones(1), weight=omega0 ** 4),
                  RowSet(t0.copy(), 0.0, (1.0,), (0.0,), np.zeros(1), weight=omega0 ** 2)],
        exact=u, test_points=np.linspace(0.0, 1.0, n_test)[:, None], placement=placement)


# ----------------------------------------------------------------------------
# the five named workloads
# ----------------------------------------------------------------------------

def config_poisson1d() -> Problem:
    """1D Poisson, 16 subdomains, K=64, 2000+2 rows, FP64 throughout."""
    return poisson1d(name="poisson1d_J16_K64_N2000")


def config_poisson2d_ml() -> Problem:
    """2D Poisson, levels 1,2,4,8,16 per dim, K=128, 400^2 + 1600 rows."""
    return poisson2d(name="poisson2d_L1-16_K128_N400")


def config_dho_ml() -> Problem:
    """DHO omega0=80, zeta=0.2, levels 1..64, K=96, 20000 + 2 rows."""
    return dho(name="dho_L1-64_K96_N20000")


def random_sine_modes(seed: int, n_modes: int = 8, kmax: int = 32):
    """f = sum_m A_m sin(k_m pi x) sin(l_m pi y), k,l ~ U{1..kmax}, A ~ N(0,1).

    Returns the modes of u (amplitudes A_m / ((k^2 + l^2) pi^2)) so that
    -Laplace u = f exactly.
    """
    rng = np.random.default_rng(np.random.SeedSequence([5, seed]))
    k = rng.integers(1, kmax + 1, size=n_modes)
    l = rng.integers(1, kmax + 1, size=n_modes)
    A = rng.standard_normal(n_modes)
    return [(float(A[m] / ((k[m] ** 2 + l[m] ** 2) * math.pi ** 2)), int(k[m]), int(l[m]))
            for m in range(n_modes)]


def config_poisson2d_large(seed: int = 0, n_side: int = 2048, levels=(1, 2, 4, 8, 16, 32, 64),
                           features: int = 64) -> Problem:
    """2D Poisson, levels 1..64 per dim, K=64, 2048^2 + 4*2048 rows, random 8-mode f."""
    modes = random_sine_modes(seed)
    return poisson2d(levels=levels, features=features, n_side=n_side, modes=modes,
                     lam=(32 * math.pi) ** 4, seed=seed,
                     name=f"poisson2d_L1-64_K64_N{n_side}_f{seed}")


@dataclasses.dataclass
class BatchSpec:
    n_sub: int
    features: int
    n_side: int
    k: int


def batch_specs(n_instances: int = 512, seed: int = 0) -> List[BatchSpec]:
    """Uneven batched instances: n_sub ~ U{2..32}, K in {32,64,128}, side ~ U{64..512}, k ~ U{1..6}."""
    rng = np.random.default_rng(np.random.SeedSequence([4, seed]))
    out = []
    for _ in range(n_instances):
        out.append(BatchSpec(n_sub=int(rng.integers(2, 33)),
                             features=int(rng.choice([32, 64, 128])),
                             n_side=int(rng.integers(64, 513)),
                             k=int(rng.integers(1, 7))))
    return out


def support_points_per_feature(P: Problem) -> float:
    """Interior collocation points that one interior subdomain of the finest
    level holds in its support, per feature: the support covers (delta / n)^dim
    of the domain box (n subdomains per dimension), for uniformly spread
    points.  Below a few, the subdomain's features are under-resolved and its
    Gram block is singular or nearly so."""
    n = P.levels[-1]
    return P.interior.points.shape[0] * min(1.0, P.delta / n) ** P.dim / P.features


def batch_instance(spec: BatchSpec, index: int, batch_seed: int = 0) -> Problem:
    """One single-level 2D Poisson instance u = sin(k pi x) sin(k pi y)."""
    return poisson2d(levels=(spec.n_sub,), features=spec.features, n_side=spec.n_side,
                     modes=[(1.0, spec.k, spec.k)], lam=(spec.k * math.pi) ** 4,
                     seed=(batch_seed << 20) + index, n_test_side=64,
                     name=f"batch{batch_seed}_{index}")


def laplace_multiscale(omegas=(4, 8, 12, 16), levels=(16,), features: int = 16,
                       delta: float = 2.9, n_grid: int = 80, n_test: int = 96, seed: int = 0,
                       weight_scale: float = 1.0, placement: str = "cell",
                       name: str = None) -> Problem:
    """§4.3 Eq. ``laplace_problem``: -Laplace u = f on [0,1]^2, u = 0 on the
    boundary, with f of Eq. ``multiscale_laplace_f``,
    f = (2 / n) sum_i (w_i pi)^2 sin(w_i pi x) sin(w_i pi y), exact solution
    u = (1 / n) sum_i sin(w_i pi x) sin(w_i pi y); the boundary condition is
    imposed by the hard-constraint ansatz with w = w_n (the largest frequency),
    so there are no boundary rows.  Collocation: the midpoints of an n_grid^2
    grid (80^2 in the baseline); test points: an n_test^2 grid.
    """
    n = len(omegas)
    modes = [(1.0 / n, w, w) for w in omegas]
    u, f = _sine_modes_2d(modes)
    xi = grid2d(midpoints(n_grid), midpoints(n_grid))
    t = np.linspace(0.0, 1.0, n_test)
    return Problem(
        name=name or f"laplace_n{n}_J{'-'.join(map(str, levels))}_K{features}",
        dim=2, lo=(0.0, 0.0), hi=(1.0, 1.0), levels=tuple(levels), delta=delta,
        features=features, seed=seed, weight_scale=weight_scale,
        interior=RowSet(xi, 0.0, (0.0, 0.0), (-1.0, -1.0), f(xi)),
        boundary=[], exact=u, test_points=grid2d(t, t), placement=placement,
        ansatz_omega=float(max(omegas)))


def helmholtz_lshape(omega: float = 8.0, k: float = 1.0, levels=(16,), features: int = 16,
                     delta: float = 2.9, n_grid: int = 80, n_long: int = 80, n_short: int = 40,
                     n_test: int = 96, seed: int = 0, weight_scale: float = 1.0,
                     placement: str = "cell", name: str = None) -> Problem:
    """§4.4 Eq. ``helmholtz_problem``: Laplace u + k^2 u = f on the L-shaped domain
    [0,1]^2 minus [0.5,1] x [0.5,1], u = g on its boundary, with the manufactured
    solution u = sin(w pi x) sin(2 w pi y) + sin(3 w pi x y) (Eq. ``helmholtz_exact``)
    and f from Eq. ``helmholtz_f``; lambda_bc = 25 w^4 (§4.4 "Physics-informed
    objective").  Interior points: the midpoints of an n_grid^2 grid over [0,1]^2
    outside the cut-out square (80^2 - 40^2 = 4800 in the baseline); boundary:
    midpoints of n_long points on each of the two long segments and n_short on
    each of the four short ones (320); test points: an n_test^2 grid over
    [0,1]^2 outside the cut-out square.  Subdomains centred in the cut-out
    square are discarded (§4.1).
    """
    wp = omega * math.pi

    def u(p):
        p = np.asarray(p)
        x, y = p[..., 0], p[..., 1]
        return np.sin(wp * x) * np.sin(2 * wp * y) + np.sin(3 * wp * x * y)

    def f(p):
        p = np.asarray(p)
        x, y = p[..., 0], p[..., 1]
        return (-5.0 * wp ** 2 * np.sin(wp * x) * np.sin(2 * wp * y)
                - 9.0 * wp ** 2 * (x * x + y * y) * np.sin(3 * wp * x * y)
                + k * k * (np.sin(wp * x) * np.sin(2 * wp * y) + np.sin(3 * wp * x * y)))

    def outside_cut(P):
        return ~((P[:, 0] > 0.5) & (P[:, 1] > 0.5))

    g = grid2d(midpoints(n_grid), midpoints(n_grid))
    xi = g[outside_cut(g)]
    ml, ms = midpoints(n_long), midpoints(n_short)
    zl, ol = np.zeros(n_long), np.ones(n_long)
    zs, os_ = np.zeros(n_short), np.ones(n_short)
    xb = np.concatenate([
        np.stack([ml, zl], 1),                     # y = 0, x in (0, 1)
        np.stack([os_, 0.5 * ms], 1),              # x = 1, y in (0, 0.5)
        np.stack([1.0 - 0.5 * ms, 0.5 * os_], 1),  # y = 0.5, x in (0.5, 1)
        np.stack([0.5 * os_, 0.5 + 0.5 * ms], 1),  # x = 0.5, y in (0.5, 1)
        np.stack([0.5 - 0.5 * ms, os_], 1),        # y = 1, x in (0, 0.5)
        np.stack([zl, 1.0 - ml], 1),               # x = 0, y in (0, 1)
    ])
    t = np.linspace(0.0, 1.0, n_test)
    gt = grid2d(t, t)
    return Problem(
        name=name or f"helmholtz_L_w{omega:g}_J{'-'.join(map(str, levels))}_K{features}",
        dim=2, lo=(0.0, 0.0), hi=(1.0, 1.0), levels=tuple(levels), delta=delta,
        features=features, seed=seed, weight_scale=weight_scale,
        interior=RowSet(xi, k * k, (0.0, 0.0), (1.0, 1.0), f(xi)),
        boundary=[RowSet(xb, 1.0, (0.0, 0.0), (0.0, 0.0), u(xb), weight=25.0 * omega ** 4)],
        exact=u, test_points=gt[outside_cut(gt)], placement=placement,
        holes=(((0.5, 0.5), (1.0, 1.0)),))


def dho_paper_baseline(seed: int = 0) -> Problem:
    """§4.2 baseline: omega0=80, beta=2, J=20, K=12, delta=2.9, R=1, 260 points.

    Subdomain centres at the interval end points ("equally spaced over the
    domain", §4.1), as in the paper's own experiments.
    """
    return dho(levels=(20,), features=12, n_interior=260, omega0=80.0, beta=2.0,
               delta=2.9, seed=seed, placement="endpoint", name="dho_paper_baseline")


CONFIGS = {
    "poisson1d": config_poisson1d,
    "poisson2d_ml": config_poisson2d_ml,
    "dho_ml": config_dho_ml,
    "poisson2d_large": config_poisson2d_large,
}
