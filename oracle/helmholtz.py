"""Discretised scattered-field Helmholtz operator on the extended domain (oracle, test infrastructure).

Follows Sec. IV-A of the paper:
  * Omega_e = Omega plus an absorbing boundary layer (ABL) of `abl` cells per side;
  * uniform grid x = (m h, n h); unknown u_{m,n} is entry n*nx + m (x fastest);
  * five-point row  (4 u_{m,n} - u_{m-1,n} - u_{m+1,n} - u_{m,n-1} - u_{m,n+1}) / h^2
                    - alpha * c_{m,n} * u_{m,n} = b_{m,n},
    with c = (k0 eta)^2 = k^2 (1 + f_d) on Omega and k^2 in the layer;
  * first-order Sommerfeld closure through ghost values u_{-1,n} = (1 + j h k_b) u_{0,n}
    (and likewise on all four sides), k_b = k the background wavenumber at the boundary.

Readings where the paper is silent or at odds with itself:
  * damping sign: the paper's time factor e^{-j w t} (Sec. II-A) makes the outgoing closure
    add -(1 + j h k)/h^2 to the diagonal (negative imaginary part).  The layer factor is
    taken with the same sign so that it absorbs: alpha = 1 + j beta (d/L)^2, giving
    Im(diag) <= 0 everywhere;
  * the layer profile ||x - P_Omega(x)||^2 / L is read dimensionless as (d/L)^2 with d the
    Euclidean distance, in fine cells, from the grid point to Omega's index box and L the
    layer width in cells;
  * the shifted-Laplacian operator K_kappa = -lap - kappa * alpha * c (Sec. IV-B) keeps the
    closure unshifted; with kappa = 1 it is A itself.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """Geometry and physics of one discretised problem (Sec. IV-A)."""
    nx_int: int
    ny_int: int
    abl: int
    h: float
    k: float
    beta: float = 0.15

    @property
    def nx(self) -> int:
        return self.nx_int + 2 * self.abl

    @property
    def ny(self) -> int:
        return self.ny_int + 2 * self.abl

    @classmethod
    def from_workload(cls, w) -> "Problem":
        return cls(w.nx_int, w.ny_int, w.abl, w.h, w.k, w.beta)


def layer_distance_sq(p: Problem, nx: int, ny: int, scale: int = 1) -> np.ndarray:
    """Squared distance, in fine cells, from the fine position (scale*i, scale*j) of each point
    of an nx-by-ny level to Omega's index box [abl, abl+nx_int-1] x [abl, abl+ny_int-1]."""
    m = scale * np.arange(nx, dtype=np.float64)
    n = scale * np.arange(ny, dtype=np.float64)
    lo_x, hi_x = p.abl, p.abl + p.nx_int - 1
    lo_y, hi_y = p.abl, p.abl + p.ny_int - 1
    dx = np.maximum(np.maximum(lo_x - m, 0.0), m - hi_x)
    dy = np.maximum(np.maximum(lo_y - n, 0.0), n - hi_y)
    return dy[:, None] ** 2 + dx[None, :] ** 2


def absorbing_factor(p: Problem, nx: int = None, ny: int = None, scale: int = 1) -> np.ndarray:
    """ABL factor alpha = 1 + j*beta*(d/L)^2 at every point of a level (Sec. IV-A, sign reading above)."""
    nx = p.nx if nx is None else nx
    ny = p.ny if ny is None else ny
    d2 = layer_distance_sq(p, nx, ny, scale)
    if p.abl == 0:
        return np.ones((ny, nx), dtype=np.complex128)
    return 1.0 + 1j * p.beta * d2 / float(p.abl) ** 2


def fine_coefficient(p: Problem, f_d: np.ndarray) -> np.ndarray:
    """c = (k0 eta)^2 on Omega_e: k^2 (1 + f_d) inside Omega, k^2 in the layer (Sec. II-A, f = k^2 f_d)."""
    c = np.full((p.ny, p.nx), p.k ** 2, dtype=np.float64)
    a = p.abl
    c[a:a + p.ny_int, a:a + p.nx_int] = p.k ** 2 * (1.0 + f_d)
    return c


def missing_neighbours(nx: int, ny: int) -> np.ndarray:
    """Number of the four stencil neighbours that fall outside the grid (0, 1 or 2)."""
    cnt = np.zeros((ny, nx), dtype=np.int64)
    cnt[:, 0] += 1
    cnt[:, -1] += 1
    cnt[0, :] += 1
    cnt[-1, :] += 1
    return cnt


def operator_diagonal(c: np.ndarray, alpha: np.ndarray, h: float, k: float,
                      shift: complex = 1.0) -> np.ndarray:
    """Diagonal of the five-point operator: 4/h^2 - shift*alpha*c, plus -(1 + j h k)/h^2 for
    each neighbour replaced by its Sommerfeld ghost value (Sec. IV-A)."""
    ny, nx = c.shape
    nmiss = missing_neighbours(nx, ny)
    return 4.0 / h ** 2 - shift * alpha * c - nmiss * (1.0 + 1j * h * k) / h ** 2


def neighbour_sum(u: np.ndarray) -> np.ndarray:
    """Sum of the four in-grid neighbours of every point (missing ones contribute 0)."""
    s = np.zeros_like(u)
    s[:, 1:] += u[:, :-1]
    s[:, :-1] += u[:, 1:]
    s[1:, :] += u[:-1, :]
    s[:-1, :] += u[1:, :]
    return s


def apply_operator(D: np.ndarray, u: np.ndarray, h: float) -> np.ndarray:
    """y = K u for the five-point operator with diagonal D: y = D*u - (sum of neighbours)/h^2."""
    return D * u - neighbour_sum(u) / h ** 2


def assemble_operator(D: np.ndarray, h: float) -> sp.csr_matrix:
    """The same operator as a sparse matrix, row n*nx + m (Sec. IV-A ordering)."""
    ny, nx = D.shape
    N = nx * ny
    idx = np.arange(N).reshape(ny, nx)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [D.ravel().astype(np.complex128)]
    off = -1.0 / h ** 2
    for (a, b) in ((idx[:, 1:], idx[:, :-1]), (idx[:, :-1], idx[:, 1:]),
                   (idx[1:, :], idx[:-1, :]), (idx[:-1, :], idx[1:, :])):
        rows.append(a.ravel())
        cols.append(b.ravel())
        vals.append(np.full(a.size, off, dtype=np.complex128))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))
