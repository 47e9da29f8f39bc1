"""Multilevel overlapping decomposition (oracle side).

§3 "Problem and model definition": levels l = 1..L, each covering the domain
with J_l overlapping subdomains.  §4.1 "Domain decomposition": a uniform
tensor grid of subdomains per level; in one dimension subdomain j has bounds
mu_j -/+ (delta/2) * (spacing), half-width sigma = (x_max - x_min) / 2, with
delta the width ratio.

Readings (the paper is silent or ambiguous):
* placement "cell" (default): centres are cell-centred,
  mu_j = lo + (j + 1/2) * Delta with Delta = (hi - lo) / n;
* placement "endpoint": centres equally spaced including both end points,
  mu_j = lo + j * Delta with Delta = (hi - lo) / (n - 1) (a single subdomain
  sits at the midpoint with Delta = hi - lo);
* the end subdomains use the same spacing Delta on their outer side, so every
  subdomain has sigma = delta * Delta / 2;
* within a level, 2-D subdomains are numbered j = j_y * n + j_x (x fastest);
* the column index of (level l, subdomain j, feature k) is
  q = sum_{m<l} J_m K + j K + k  (§3 "Indexing conventions", 0-based here).

Discarding (§4.1: "we discard rectangular subdomains outside of the L-shaped
domain", for the L-shaped domain of §4.4): a problem may cut boxes (holes) out
of its domain; a subdomain is discarded when its centre lies strictly inside a
hole, a face of the hole that lies on the domain box's boundary counting as
part of the hole (reading: the paper does not say how "outside" is decided;
with the baseline's 16 x 16 grid this discards exactly the 8 x 8 subdomains it
reports, for cell-centred and for end-point centres).  Kept subdomains keep their order and are numbered consecutively;
their random parameters stay those of their full-grid column.

Parity pinned through the window tests (partition of unity, support) and the
closed-form column counts in tests/test_oracle_windows.py; discarding by the
192-subdomain count of §4.4 and the partition of unity over kept subdomains.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np


@dataclass
class Level:
    n: int                      # subdomains per dimension
    mu: List[np.ndarray]        # per dimension: centres, shape (n,)
    sigma: List[float]          # per dimension: half-width
    col_offset: int             # first column index of this level
    n_sub: int                  # J_l = n ** dim (the full grid)
    keep: np.ndarray = None     # (J_l,) bool: subdomain kept (not in a hole)
    col_first: np.ndarray = None  # (J_l,) first column of subdomain j, -1 if discarded
    param_offset: int = 0       # first full-grid column of this level (parameter draws)


def build_levels(dim: int, lo, hi, levels, delta: float, K: int,
                 placement: str = "cell", holes=()) -> List[Level]:
    out = []
    off = 0
    poff = 0
    for n in levels:
        mus, sigs = [], []
        for i in range(dim):
            if placement == "cell":
                D = (hi[i] - lo[i]) / n
                mus.append(lo[i] + (np.arange(n, dtype=np.float64) + 0.5) * D)
            elif placement == "endpoint":
                if n == 1:
                    D = hi[i] - lo[i]
                    mus.append(np.array([0.5 * (lo[i] + hi[i])]))
                else:
                    D = (hi[i] - lo[i]) / (n - 1)
                    mus.append(lo[i] + np.arange(n, dtype=np.float64) * D)
            else:
                raise ValueError(f"unknown placement {placement!r}")
            sigs.append(delta * D / 2.0)
        J = n ** dim
        lev = Level(n=n, mu=mus, sigma=sigs, col_offset=off, n_sub=J)
        keep = np.ones(J, dtype=bool)
        for j in range(J):
            ji = subdomain_multi_index(lev, dim, j)
            centre = [mus[i][ji[i]] for i in range(dim)]
            for hlo, hhi in holes:
                if all(_in_hole(centre[i], hlo[i], hhi[i], lo[i], hi[i]) for i in range(dim)):
                    keep[j] = False
        lev.keep = keep
        lev.col_first = np.where(keep, off + (np.cumsum(keep) - 1) * K, -1)
        lev.param_offset = poff
        out.append(lev)
        off += int(keep.sum()) * K
        poff += J * K
    return out


def _in_hole(c: float, hlo: float, hhi: float, lo: float, hi: float) -> bool:
    """Centre coordinate c inside the hole's extent along one axis: strictly
    between its faces, a face that lies on the domain box's boundary counting
    as part of the hole (a centre on the box edge beyond the cut is outside
    the domain too)."""
    above = c > hlo or (hlo == lo and c == lo)
    below = c < hhi or (hhi == hi and c == hi)
    return above and below


def n_columns(problem) -> int:
    """N_Phi = K x (subdomains kept over all levels)."""
    levels = build_levels(problem.dim, problem.lo, problem.hi, problem.levels, problem.delta,
                          problem.features, problem.placement, getattr(problem, "holes", ()))
    return sum(int(lev.keep.sum()) for lev in levels) * problem.features


def subdomain_multi_index(level: Level, dim: int, j: int) -> Tuple[int, ...]:
    """Linear subdomain index j -> (j_x, j_y, ...) with x fastest."""
    idx = []
    for _ in range(dim):
        idx.append(j % level.n)
        j //= level.n
    return tuple(idx)


def all_subdomains(level: Level, dim: int):
    """Iterate (j, (j_x, j_y, ...)) over the level in linear order."""
    for j, rev in enumerate(itertools.product(range(level.n), repeat=dim)):
        yield j, tuple(reversed(rev))
