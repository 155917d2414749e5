"""Incident fields, right-hand sides, sensor sampling and the data-term gradient (oracle, test
infrastructure).

Follows Sec. II-A (plane wave u_in = u0 e^{j<k,x>}, scattered-field equation
-lap u_sc - k0^2 eta^2 u_sc = f u_in with f = k0^2 (eta^2 - eta_b^2)), Sec. IV-A (truncation of
the solution from Omega_e to Omega) and Sec. V (quadratic data term, Prop. 1).

In the dimensionless contrast f_d = (n/n_b)^2 - 1 used here, f = k^2 f_d with k = k0 eta_b.
The sensor map samples u_sc on receiver grid points (an index set S) instead of propagating it
with a Green's function; for L = 1/2 sum_q ||S u_sc,q - y_q||^2, Prop. 1's linearisation
d u_q = A^{-1} diag(u_q) df (u_q = u_in,q + u_sc,q the total field) and the complex symmetry
A^T = A give
    dL/df_d = k^2 sum_q Re(z_q * u_q)   on Omega,   with   A z_q = S^T conj(S u_sc,q - y_q).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .helmholtz import Problem, absorbing_factor, fine_coefficient, operator_diagonal, apply_operator, assemble_operator
from .multigrid import Preconditioner
from .krylov import fgmres, bicgstab


def incident_field(p: Problem, theta: float) -> np.ndarray:
    """u_in = exp(j k (x cos(theta) + y sin(theta))) at x = m h, y = n h (Sec. II-A, Sec. IV-A), u0 = 1."""
    x = p.h * np.arange(p.nx, dtype=np.float64)
    y = p.h * np.arange(p.ny, dtype=np.float64)
    phase = p.k * (np.cos(theta) * x[None, :] + np.sin(theta) * y[:, None])
    return np.exp(1j * phase)


def embed(p: Problem, a_int: np.ndarray) -> np.ndarray:
    """Place an interior array [ny_int][nx_int] into Omega_e, zero in the layer."""
    out = np.zeros((p.ny, p.nx), dtype=a_int.dtype)
    a = p.abl
    out[a:a + p.ny_int, a:a + p.nx_int] = a_int
    return out


def rhs(p: Problem, f_d: np.ndarray, theta: float) -> np.ndarray:
    """b = f u_in = k^2 f_d u_in on Omega_e (f_d = 0 in the layer) (Sec. II-A)."""
    return p.k ** 2 * embed(p, f_d) * incident_field(p, theta)


def crop(p: Problem, u: np.ndarray) -> np.ndarray:
    """Truncate a field on Omega_e to Omega (Sec. IV-A)."""
    a = p.abl
    return u[..., a:a + p.ny_int, a:a + p.nx_int]


def sample(u: np.ndarray, receivers: np.ndarray) -> np.ndarray:
    """S u: the field at the receiver grid points (flat indices on Omega_e)."""
    return u.reshape(u.shape[:-2] + (-1,))[..., receivers]


def misfit(u_rec: np.ndarray, y: np.ndarray):
    """Residual r = S u - y and the quadratic data term 1/2 sum ||r||^2 (Sec. V)."""
    r = u_rec - y
    return r, 0.5 * float(np.sum(np.abs(r) ** 2))


def gradient_from_adjoint(p: Problem, z: np.ndarray, u_tot: np.ndarray) -> np.ndarray:
    """g = k^2 sum_q Re(z_q u_q) restricted to Omega (Prop. 1 with dA = -k^2 diag(df_d))."""
    return p.k ** 2 * crop(p, np.real(z * u_tot)).sum(axis=0)


def direct_solve(p: Problem, D: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Exact discrete solution A^{-1} b by a sparse LU (SuperLU)."""
    A = assemble_operator(D, p.h).tocsc()
    return spla.spsolve(A, b.ravel()).reshape(b.shape)


class MGHSolver:
    """The paper's MGH solver on one contrast: operator A, shifted-Laplacian MG preconditioner and
    a Krylov method, plus the forward map and the data-term gradient."""

    def __init__(self, p: Problem, f_d: np.ndarray, levels: int, nu1, nu2,
                 omega: float = 0.8, shift: complex = 1.0 + 0.5j, restart: int = 20,
                 tol: float = 1e-6, maxit: int = 5000, cycle_type: int = 1, krylov: str = "gmres"):
        self.p = p
        self.f_d = f_d
        self.c = fine_coefficient(p, f_d)
        self.alpha = absorbing_factor(p)
        self.D = operator_diagonal(self.c, self.alpha, p.h, p.k, 1.0)       # A (unshifted)
        self.M = Preconditioner(p, self.c, levels, nu1, nu2, omega, shift, cycle_type)
        self.restart, self.tol, self.maxit, self.krylov = restart, tol, maxit, krylov

    def apply_A(self, u: np.ndarray) -> np.ndarray:
        return apply_operator(self.D, u, self.p.h)

    def solve(self, b: np.ndarray, tol: float = None, x0: np.ndarray = None):
        tol = self.tol if tol is None else tol
        if self.krylov == "bicgstab":
            return bicgstab(self.apply_A, self.M, b, tol, self.maxit, x0)
        return fgmres(self.apply_A, self.M, b, tol, self.restart, self.maxit, x0)

    def forward(self, thetas, tol: float = None):
        """u_sc for every illumination angle; returns ([B][ny][nx] complex128, [SolveInfo])."""
        us, infos = [], []
        for th in thetas:
            u, info = self.solve(rhs(self.p, self.f_d, float(th)), tol)
            us.append(u)
            infos.append(info)
        return np.stack(us), infos

    def gradient(self, thetas, receivers: np.ndarray, y: np.ndarray, tol: float = None):
        """Loss 1/2 sum_q ||S u_sc,q - y_q||^2 and its gradient in f_d on Omega (Prop. 1)."""
        u_sc, _ = self.forward(thetas, tol)
        r, loss = misfit(sample(u_sc, receivers), y)
        g = np.zeros((self.p.ny_int, self.p.nx_int))
        for q, th in enumerate(thetas):
            G = np.zeros(self.p.ny * self.p.nx, dtype=np.complex128)
            np.add.at(G, receivers, np.conj(r[q]))
            z, _ = self.solve(G.reshape(self.p.ny, self.p.nx), tol)
            u_tot = u_sc[q] + incident_field(self.p, float(th))
            g += gradient_from_adjoint(self.p, z[None], u_tot[None])
        return loss, g, u_sc
