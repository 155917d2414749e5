"""Shifted-Laplacian multigrid preconditioner (oracle, test infrastructure).

Follows Sec. III (damped Jacobi, eq. dampedJ; MG cycle, Alg. 2) and Sec. IV-C (full-weighting
restriction, bilinear prolongation as the adjoint of R, re-discretised coarse operators with
the full-weighted coefficient k0^2 eta^2 and its boundary ring reset to k0^2 eta_b^2, coarsest
level solved exactly).

Reading for even grid sizes (the paper's indices assume an odd number of points): a level of
n points coarsens to n_c = floor((n-1)/2) + 1 points, coarse index i sitting on fine index 2i.
R reads fine samples 2i-1, 2i, 2i+1 and counts out-of-range samples as 0; P = 4 R^T, so a
fine point whose second coarse neighbour is out of range receives only the in-range half.
Coarse boundary points stay unknowns (the Robin closure makes them so).  The coarse layer
factor alpha is evaluated at each coarse point's fine position, with distances in fine cells,
and the same shift kappa is used on every level.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np
import scipy.linalg as sla

from .helmholtz import Problem, absorbing_factor, operator_diagonal, apply_operator, assemble_operator


def coarse_size(n: int) -> int:
    """Number of coarse points for n fine points: coarse i <-> fine 2i."""
    return (n - 1) // 2 + 1


def restrict(r: np.ndarray) -> np.ndarray:
    """Full weighting (Sec. IV-C): r2h[i,j] = (4 r[2i,2j] + 2 (edge neighbours) + (corner neighbours)) / 16,
    with fine samples outside the grid counted as 0.  Arrays are [n][m] (y rows, x columns)."""
    ny, nx = r.shape
    nyc, nxc = coarse_size(ny), coarse_size(nx)
    rp = np.zeros((ny + 2, nx + 2), dtype=r.dtype)   # rp[n+1, m+1] = r[n, m]; zeros around
    rp[1:-1, 1:-1] = r

    def at(dn, dm):  # samples r[2j+dn, 2i+dm] for all coarse (j, i)
        return rp[1 + dn:1 + dn + 2 * nyc:2, 1 + dm:1 + dm + 2 * nxc:2]

    centre = at(0, 0)
    edges = at(0, -1) + at(0, 1) + at(-1, 0) + at(1, 0)
    corners = at(-1, -1) + at(-1, 1) + at(1, -1) + at(1, 1)
    return (4.0 * centre + 2.0 * edges + corners) / 16.0


def prolong(ec: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Bilinear prolongation (Sec. IV-C), the four parity cases of the fine index (m, n);
    coarse samples outside the coarse grid are 0."""
    nyc, nxc = ec.shape
    assert nyc == coarse_size(ny) and nxc == coarse_size(nx)
    ep = np.zeros((nyc + 1, nxc + 1), dtype=ec.dtype)
    ep[:nyc, :nxc] = ec
    e = np.zeros((ny, nx), dtype=ec.dtype)
    ne, no = (ny + 1) // 2, ny // 2          # even / odd fine rows
    me, mo = (nx + 1) // 2, nx // 2          # even / odd fine columns
    e[0::2, 0::2] = ep[:ne, :me]
    e[0::2, 1::2] = 0.5 * (ep[:ne, :mo] + ep[:ne, 1:mo + 1])
    e[1::2, 0::2] = 0.5 * (ep[:no, :me] + ep[1:no + 1, :me])
    e[1::2, 1::2] = 0.25 * (ep[:no, :mo] + ep[:no, 1:mo + 1] + ep[1:no + 1, :mo] + ep[1:no + 1, 1:mo + 1])
    return e


def restrict_coefficient(c: np.ndarray, k: float) -> np.ndarray:
    """Coarse k0^2 eta^2: full weighting of the fine one, then the outermost ring set to the
    background value k0^2 eta_b^2 = k^2 (Sec. IV-C)."""
    cc = restrict(c)
    cc[0, :] = k ** 2
    cc[-1, :] = k ** 2
    cc[:, 0] = k ** 2
    cc[:, -1] = k ** 2
    return cc


@dataclass
class Level:
    nx: int
    ny: int
    h: float
    scale: int          # fine cells per coarse cell, 2^l
    c: np.ndarray       # real k0^2 eta^2 on this level
    D: np.ndarray       # complex diagonal of K_kappa on this level


def build_hierarchy(p: Problem, c_fine: np.ndarray, levels: int, shift: complex) -> List[Level]:
    """Levels 0..levels-1 of K_kappa, re-discretised with spacing 2^l h (Sec. IV-C)."""
    out = []
    c, nx, ny, h, s = c_fine, p.nx, p.ny, p.h, 1
    for l in range(levels):
        alpha = absorbing_factor(p, nx, ny, s)
        out.append(Level(nx, ny, h, s, c, operator_diagonal(c, alpha, h, p.k, shift)))
        if l + 1 < levels:
            c = restrict_coefficient(c, p.k)
            nx, ny, h, s = coarse_size(nx), coarse_size(ny), 2.0 * h, 2 * s
    return out


def jacobi(lv: Level, b: np.ndarray, v: np.ndarray, omega: float) -> np.ndarray:
    """One damped Jacobi step v <- v - omega D^{-1} (K v - b) (Sec. III, eq. dampedJ)."""
    return v - omega * (apply_operator(lv.D, v, lv.h) - b) / lv.D


class CoarseSolver:
    """Exact solve on the coarsest level (Alg. 2, Sec. IV-C) by LAPACK LU with partial pivoting."""

    def __init__(self, lv: Level):
        A = assemble_operator(lv.D, lv.h).toarray()
        self.lu = sla.lu_factor(A)
        self.shape = (lv.ny, lv.nx)

    def __call__(self, b: np.ndarray) -> np.ndarray:
        return sla.lu_solve(self.lu, b.ravel()).reshape(self.shape)


def _sweeps(nu, l: int) -> int:
    """Sweeps on level l: nu is one count for every level or a sequence indexed by level (the
    counts need not be equal across levels, Sec. III after Alg. 2)."""
    return int(nu) if np.isscalar(nu) else int(nu[l])


def mg_cycle(hier: List[Level], coarse: CoarseSolver, l: int, b: np.ndarray, v: np.ndarray,
             nu1, nu2, omega: float, cycle_type: int = 1) -> np.ndarray:
    """MGCycle of Alg. 2 (V-cycle for cycle_type=1, W-cycle for 2) on level l; nu1 / nu2 are
    counts or per-level sequences."""
    lv = hier[l]
    if l == len(hier) - 1:                       # coarsest level: solve exactly
        return coarse(b)
    for _ in range(_sweeps(nu1, l)):             # nu1 pre-relaxations
        v = jacobi(lv, b, v, omega)
    r = b - apply_operator(lv.D, v, lv.h)        # residual
    rc = restrict(r)                             # restrict to the coarse problem
    ec = np.zeros_like(rc)
    for _ in range(cycle_type):                  # CycleType recursive calls
        ec = mg_cycle(hier, coarse, l + 1, rc, ec, nu1, nu2, omega, cycle_type)
    v = v + prolong(ec, lv.ny, lv.nx)            # coarse-grid correction
    for _ in range(_sweeps(nu2, l)):             # nu2 post-relaxations
        v = jacobi(lv, b, v, omega)
    return v


class Preconditioner:
    """K_MG^{-1}: one MG cycle with zero initial guess applied to K_kappa (Alg. 3, steps 9 and 14)."""

    def __init__(self, p: Problem, c_fine: np.ndarray, levels: int, nu1, nu2,
                 omega: float, shift: complex, cycle_type: int = 1):
        self.hier = build_hierarchy(p, c_fine, levels, shift)
        self.coarse = CoarseSolver(self.hier[-1])
        self.nu1, self.nu2, self.omega, self.cycle_type = nu1, nu2, omega, cycle_type

    def __call__(self, b: np.ndarray) -> np.ndarray:
        return mg_cycle(self.hier, self.coarse, 0, b, np.zeros_like(b), self.nu1, self.nu2,
                        self.omega, self.cycle_type)
