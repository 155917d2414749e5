"""Pins of the oracle's flexible GMRES with deflated restarting (oracle.krylov.fgmres_dr, Morgan
2002; flexible form of Giraud et al. 2010): the method the strong-scattering workload needs with a
single-precision cycle, where ordinary restarts stagnate."""
from dataclasses import replace

import numpy as np

import oracle as O
import workloads as W
from oracle.krylov import deflated_restart, fgmres, fgmres_dr, harmonic_ritz


def _small(seed=5, n=24, levels=3):
    w = W.small_workload(n_int=n, abl=4, seed=seed, levels=levels)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    return p, f, O.MGHSolver(p, f, levels=levels, nu1=1, nu2=1, tol=1e-30)


def test_without_deflation_it_is_restarted_fgmres():
    """k = 0 keeps only the residual: three cycles equal three cycles of FGMRES(m)."""
    p, f, s = _small()
    b = O.rhs(p, f, 0.4)
    x_dr, info_dr = fgmres_dr(s.apply_A, s.M, b, 1e-30, 6, 0, 18)
    x_gm, info_gm = fgmres(s.apply_A, s.M, b, 1e-30, 6, 18)
    assert info_dr.iterations == info_gm.iterations == 18
    assert np.linalg.norm(x_dr - x_gm) <= 1e-9 * np.linalg.norm(x_gm)


def _arnoldi(s, b, m):
    """m steps of Arnoldi on A M^{-1} from b (classical Gram-Schmidt, two passes)."""
    n = b.size
    V = np.zeros((n, m + 1), complex)
    Z = np.zeros((n, m), complex)
    H = np.zeros((m + 1, m), complex)
    beta = np.linalg.norm(b)
    V[:, 0] = b.ravel() / beta
    for j in range(m):
        Z[:, j] = s.M(V[:, j].reshape(b.shape)).ravel()
        w = s.apply_A(Z[:, j].reshape(b.shape)).ravel()
        for _ in range(2):
            h = V[:, :j + 1].conj().T @ w
            w -= V[:, :j + 1] @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, Z, H, beta


def test_harmonic_ritz_vectors_solve_their_defining_problem():
    """Hbar^H Hbar g = theta H_m^H g for each returned g, theta its harmonic Ritz value; the
    returned ones have the smallest |theta| of all m."""
    p, f, s = _small(seed=6)
    V, Z, H, _ = _arnoldi(s, O.rhs(p, f, 0.2), 10)
    G = harmonic_ritz(H, 4)
    Hm = H[:10, :]
    thetas_all = np.linalg.eigvals(np.linalg.solve(Hm.conj().T, H.conj().T @ H))
    for i in range(4):
        g = G[:, i]
        lhs = H.conj().T @ (H @ g)
        rhs = Hm.conj().T @ g
        theta = (rhs.conj() @ lhs) / (rhs.conj() @ rhs)
        assert np.linalg.norm(lhs - theta * rhs) <= 1e-9 * np.linalg.norm(lhs)
        assert abs(theta) <= np.sort(np.abs(thetas_all))[3] * (1 + 1e-9)


def test_deflated_restart_keeps_the_arnoldi_relation_and_the_residual():
    """After the restart, A Z_new = V_new H_new (the relation flexible GMRES needs), V_new has
    orthonormal columns, and V_new g_new is the residual of the cycle's iterate."""
    p, f, s = _small(seed=7)
    b = O.rhs(p, f, -0.3)
    m, k = 10, 4
    V, Z, H, beta = _arnoldi(s, b, m)
    g = np.zeros(m + 1, complex)
    g[0] = beta
    y = np.linalg.lstsq(H, g, rcond=None)[0]
    x = (Z @ y).reshape(b.shape)
    c = g - H @ y
    Vn, Zn, Hn, gn = deflated_restart(V, Z, H, c, k)
    AZ = np.stack([s.apply_A(Zn[:, i].reshape(b.shape)).ravel() for i in range(k)], axis=1)
    assert np.linalg.norm(AZ - Vn @ Hn) <= 1e-10 * np.linalg.norm(AZ)
    assert np.linalg.norm(Vn.conj().T @ Vn - np.eye(k + 1)) <= 1e-12
    r = (b - s.apply_A(x)).ravel()
    assert np.linalg.norm(Vn @ gn - r) <= 1e-10 * np.linalg.norm(r)


def test_deflated_restarts_beat_plain_restarts_on_the_strong_scattering_recipe():
    """On the cell recipe at 128^2 + 8 (n/n_b to 1.5, 12 points per wavelength) FGMRES-DR(8, 4)
    reaches the direct solution in fewer steps than FGMRES(8) (measured 1,814)."""
    w = replace(W.WORKLOADS["cell1120"], name="cell128", nx_int=128, ny_int=128, abl=8, levels=4,
                shift_im=1.0, krylov="fgmres")
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    s = O.MGHSolver(p, f, w.levels, 2, 2, 0.8, complex(w.shift_re, w.shift_im), 8, 1e-8, maxit=4000)
    b = O.rhs(p, f, 0.3)
    x_dr, info_dr = fgmres_dr(s.apply_A, s.M, b, 1e-8, 8, 4, 4000)
    _, info_gm = s.solve(b)
    assert info_dr.converged and info_gm.converged
    assert info_dr.iterations < info_gm.iterations, (info_dr.iterations, info_gm.iterations)
    ref = O.direct_solve(p, s.D, b)
    assert np.linalg.norm(x_dr - ref) <= 1e-5 * np.linalg.norm(ref)
