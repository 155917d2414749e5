"""Krylov solvers (oracle, test infrastructure).

* fgmres: right-preconditioned flexible GMRES(m) -- the textbook method of Saad & Schultz
  (1986) with the flexible variant of Saad (1993), modified Gram-Schmidt Arnoldi and complex
  Givens rotations for the Hessenberg least-squares problem.  With a fixed linear
  preconditioner it is ordinary right-preconditioned GMRES.  The iterate is accepted only
  when the true residual ||b - A x|| / ||b|| <= tol (the relative stopping rule of Sec. VI);
  the Givens estimate only decides when to leave an Arnoldi cycle early.
* bicgstab: the paper's preconditioned Bi-CGSTAB, Alg. 3, with the relative stopping rule.
* sstep_cycle: one restart cycle of FGMRES(m) in s-step form (Chronopoulos & Gear 1989; Hoemmen
  2010): the monomial basis v_{k+1} = A M^{-1} v_k is orthogonalised at the end of the cycle by
  the Cholesky factor of its Gram matrix.  In exact arithmetic it returns the iterate of one
  Arnoldi cycle of fgmres; the CUDA path's default mixed engine is built on this identity.
* fgmres_dr: flexible GMRES with deflated restarting (Morgan 2002; Giraud et al. 2010), which
  keeps k harmonic Ritz vectors across restarts: the method for problems on which ordinary
  restarts stagnate (the strong-scattering workload).
* idrs: IDR(s) with biorthogonalisation (Sonneveld & van Gijzen 2008; van Gijzen & Sonneveld
  2011), the short-recurrence family Alg. 3 belongs to (s = 1 with the shadow vector r_0 is
  Bi-CGSTAB).

Iterations are counted as preconditioner applications (Arnoldi steps for GMRES).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np


@dataclass
class SolveInfo:
    converged: bool = False
    iterations: int = 0
    restarts: int = 0
    rel_residual: float = float("inf")
    history: List[float] = field(default_factory=list)   # Givens / true residual estimates


def _dot(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = a^H b."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def _norm(a: np.ndarray) -> float:
    return float(np.sqrt(np.vdot(a.ravel(), a.ravel()).real))


def givens(a: complex, b: complex):
    """Rotation [[c, s], [-conj(s), c]] (c real) mapping (a, b) to (r, 0)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, 1.0 + 0.0j
    rho = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / rho
    s = (a / abs(a)) * np.conj(b) / rho
    return c, s


def fgmres(apply_A: Callable, apply_M: Callable, b: np.ndarray, tol: float, restart: int,
           maxit: int, x0: np.ndarray = None):
    """Solve A x = b with right-preconditioned FGMRES(restart); returns (x, SolveInfo)."""
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        info.converged, info.rel_residual = True, 0.0
        return np.zeros_like(b), info
    m = restart
    while True:
        r = b - apply_A(x)
        beta = _norm(r)
        info.rel_residual = beta / bnorm
        info.history.append(info.rel_residual)
        if info.rel_residual <= tol:
            info.converged = True
            return x, info
        if info.iterations >= maxit:
            return x, info
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        j_end = 0
        for j in range(m):
            Z.append(apply_M(V[j]))                  # z_j = M^{-1} v_j
            w = apply_A(Z[j])
            for i in range(j + 1):                   # modified Gram-Schmidt
                H[i, j] = _dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = _norm(w)
            info.iterations += 1
            for i in range(j):                       # previous rotations on column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            j_end = j + 1
            est = abs(g[j + 1]) / bnorm
            info.history.append(est)
            breakdown = H[j, j] == 0 or _norm(w) == 0.0
            if est <= tol or info.iterations >= maxit or breakdown:
                break
            V.append(w / _norm(w))
        # back substitution for the upper-triangular j_end x j_end system
        y = np.zeros(j_end, dtype=np.complex128)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:j_end], y[i + 1:j_end])) / H[i, i]
        for i in range(j_end):
            x = x + y[i] * Z[i]
        info.restarts += 1


def bicgstab(apply_A: Callable, apply_M: Callable, b: np.ndarray, tol: float, maxit: int,
             x0: np.ndarray = None):
    """Preconditioned Bi-CGSTAB of Alg. 3 (MG cycles at steps 9 and 14), relative stopping rule."""
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        info.converged, info.rel_residual = True, 0.0
        return np.zeros_like(b), info
    r = b - apply_A(x)
    r_hat = r.copy()
    rho_prev, alpha, sigma = 1.0 + 0j, 1.0 + 0j, 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    while info.iterations < maxit:
        rho = _dot(r_hat, r)
        beta = (rho / rho_prev) * (alpha / sigma)
        p = r + beta * (p - sigma * v)
        y = apply_M(p)
        v = apply_A(y)
        alpha = rho / _dot(r_hat, v)
        hvec = x + alpha * y
        s = r - alpha * v
        z = apply_M(s)
        t = apply_A(z)
        sigma = _dot(t, s) / _dot(t, t)
        x = hvec + sigma * z
        r = s - sigma * t
        rho_prev = rho
        info.iterations += 2
        info.rel_residual = _norm(r) / bnorm
        info.history.append(info.rel_residual)
        if info.rel_residual <= tol:
            true_rel = _norm(b - apply_A(x)) / bnorm
            info.rel_residual = true_rel
            if true_rel <= tol:
                info.converged = True
                break
    return x, info


def sstep_cycle(apply_A: Callable, apply_M: Callable, b: np.ndarray, x: np.ndarray, m: int,
                gram: Callable = None) -> np.ndarray:
    """One cycle of FGMRES(m) in s-step form from the iterate x; returns the new iterate.

    gram(Vm) returns the Gram matrix Vm^H Vm of the N x (m+1) basis; the default forms it in FP64.
    A caller may pass a rounded evaluation to study how much accuracy the cycle needs in it.

    v_0 = r / ||r||, z_k = M^{-1} v_k, w_k = A z_k, v_{k+1} = w_k / ||w_k||.  With V = [v_0 .. v_m]
    and V^H V = R^H R (Cholesky, R upper), A z_k = ||w_k|| v_{k+1} and r = ||r|| v_0 give
    r - A Z y = V (||r|| e_0 - [0; diag(||w||) y]), so ||r - A Z y|| = ||R (...)||: the cycle's
    least-squares problem has the matrix R[:, 1:] diag(||w||) and the right-hand side ||r|| R[:, 0].
    """
    r = b - apply_A(x)
    beta = _norm(r)
    V = [r / beta]
    Z, wn = [], []
    for k in range(m):
        Z.append(apply_M(V[k]))
        w = apply_A(Z[k])
        wn.append(_norm(w))
        V.append(w / wn[k])
    Vm = np.stack([v.reshape(-1) for v in V], axis=1)          # N x (m+1)
    G = Vm.conj().T @ Vm if gram is None else gram(Vm)
    R = np.linalg.cholesky(G).conj().T                          # G = R^H R
    H = R[:, 1:] * np.asarray(wn)[None, :]
    y = np.linalg.lstsq(H, beta * R[:, 0], rcond=None)[0]
    x_new = x.astype(np.complex128).copy()
    for k in range(m):
        x_new = x_new + y[k] * Z[k]
    return x_new


def harmonic_ritz(Hbar: np.ndarray, k: int) -> np.ndarray:
    """The k harmonic Ritz vectors of smallest harmonic Ritz value modulus of an (m+1) x m
    Arnoldi matrix Hbar: the eigenvectors g of H_m + |h_{m+1,m}|^2 f e_m^T with H_m^H f = e_m
    (Morgan 2002), i.e. the solutions of Hbar^H Hbar g = theta H_m^H g.  Returns m x k."""
    m = Hbar.shape[1]
    Hm = Hbar[:m, :]
    em = np.zeros(m)
    em[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, em)
    T = Hm + abs(Hbar[m, m - 1]) ** 2 * np.outer(f, em)
    theta, G = np.linalg.eig(T)
    idx = np.argsort(np.abs(theta))[:k]
    return G[:, idx]


def deflated_restart(V: np.ndarray, Z: np.ndarray, H: np.ndarray, c: np.ndarray, k: int):
    """The state a deflated restart carries into the next cycle, from the cycle's V (n x (m+1)),
    Z (n x m), Hbar ((m+1) x m) with A Z = V Hbar, and the residual coefficients c (r = V c):
    P = [[G_k; 0], c] orthonormalised (G_k the k harmonic Ritz vectors), V P, Z P_k, P^H Hbar P_k
    and P^H c.  Returns (V_new n x (k+1), Z_new n x k, H_new (k+1) x k, g_new k+1)."""
    m = H.shape[1]
    P = np.zeros((m + 1, k + 1), dtype=np.complex128)
    if k > 0:
        P[:m, :k] = harmonic_ritz(H, k)
    P[:, k] = c
    Q, _ = np.linalg.qr(P)
    return V @ Q, Z @ Q[:m, :k], Q.conj().T @ H @ Q[:m, :k], Q.conj().T @ c


def fgmres_dr(apply_A: Callable, apply_M: Callable, b: np.ndarray, tol: float, m: int, k: int,
              maxit: int, x0: np.ndarray = None):
    """Right-preconditioned flexible GMRES(m) with deflated restarting (GMRES-DR of Morgan 2002 in
    the flexible form of Giraud, Gratton, Pinel & Vasseur 2010); returns (x, SolveInfo).

    A cycle runs Arnoldi from column j0 to m - 1 (classical Gram-Schmidt with a second pass) on
    z_j = M^{-1} v_j, keeping A Z = V Hbar, and takes the least-squares correction x += Z y.  The
    next cycle keeps the k harmonic Ritz vectors of smallest modulus: with P = [[g_1 .. g_k; 0], c]
    orthonormalised (c = g - Hbar y, the coefficients of the residual in V), V <- V P, Z <- Z P_k,
    Hbar <- P^H Hbar P_k and g <- P^H c, so that the relation A Z = V Hbar and r = V g carry over
    and Arnoldi continues at column k.  With k = 0 it is FGMRES(m) with ordinary restarts.  The
    iterate is accepted on the true residual ||b - A x|| <= tol ||b||, checked after every cycle;
    steps count preconditioner applications."""
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        info.converged, info.rel_residual = True, 0.0
        return np.zeros_like(b), info
    shape, n = b.shape, b.size
    r = (b - apply_A(x)).ravel()
    beta = np.linalg.norm(r)
    info.rel_residual = beta / bnorm
    if info.rel_residual <= tol:
        info.converged = True
        return x, info
    V = np.zeros((n, m + 1), dtype=np.complex128)
    Z = np.zeros((n, m), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    V[:, 0] = r / beta
    g[0] = beta
    j0 = 0
    while True:
        for j in range(j0, m):
            Z[:, j] = apply_M(V[:, j].reshape(shape)).ravel()
            w = apply_A(Z[:, j].reshape(shape)).ravel()
            for _ in range(2):
                h = V[:, :j + 1].conj().T @ w
                w = w - V[:, :j + 1] @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / H[j + 1, j]
            info.iterations += 1
        y = np.linalg.lstsq(H, g, rcond=None)[0]
        x = x + (Z @ y).reshape(shape)
        c = g - H @ y
        info.restarts += 1
        info.rel_residual = _norm(b - apply_A(x)) / bnorm
        info.history.append(info.rel_residual)
        if info.rel_residual <= tol:
            info.converged = True
            return x, info
        if info.iterations >= maxit:
            return x, info
        V_new, Z_new, H_new, g_new = deflated_restart(V, Z, H, c, k)
        V[:] = 0
        Z[:] = 0
        H[:] = 0
        g[:] = 0
        V[:, :k + 1] = V_new
        Z[:, :k] = Z_new
        H[:k + 1, :k] = H_new
        g[:k + 1] = g_new
        j0 = k

def idrs(apply_A: Callable, apply_M: Callable, b: np.ndarray, tol: float, s: int, maxit: int,
         x0: np.ndarray = None, shadow: np.ndarray = None, kappa: float = 0.7, seed: int = 0):
    """Right-preconditioned IDR(s) with biorthogonalisation (induced dimension reduction:
    Sonneveld & van Gijzen 2008; the biorthogonal variant of van Gijzen & Sonneveld 2011).

    Residuals are driven into a sequence of shrinking spaces G_j orthogonal to an s-dimensional
    shadow space P (random orthonormal unless `shadow` is given, n x s).  Each outer step makes s
    intermediate residuals with update directions U (preconditioned) and G = A U kept biorthogonal
    to P, then one dimension-reduction step r <- r - omega A M^{-1} r with omega the local
    minimal-residual choice, increased to keep |cos(t, r)| >= kappa ("maintaining the
    convergence"; kappa = 0 keeps the plain minimal residual).  Recurrences are short: storage is
    2s + 2 vectors, and each step costs one preconditioner application and one operator product.
    The iterate is accepted on the true residual ||b - A x|| <= tol ||b||; iterations count
    preconditioner applications; history holds the relative recursive residual after every
    dimension-reduction step.  With s = 1 and the shadow vector r_0 it is Bi-CGSTAB."""
    info = SolveInfo()
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        info.converged, info.rel_residual = True, 0.0
        return np.zeros_like(b), info
    shape, n = b.shape, b.size
    xr = x.ravel().astype(np.complex128)
    r = (b - apply_A(x)).ravel()
    if shadow is None:
        rng = np.random.default_rng(seed)
        P = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
        P, _ = np.linalg.qr(P)
    else:
        P = np.asarray(shadow, dtype=np.complex128).reshape(n, s)
    G = np.zeros((n, s), dtype=np.complex128)
    U = np.zeros((n, s), dtype=np.complex128)
    Ms = np.eye(s, dtype=np.complex128)     # M_s = P^H G, lower triangular after biorthogonalisation
    omega = 1.0 + 0.0j

    def accept():
        true_rel = _norm(b - apply_A(xr.reshape(shape))) / bnorm
        info.rel_residual = true_rel
        return true_rel <= tol

    while info.iterations < maxit:
        f = P.conj().T @ r
        for k in range(s):
            # v = r - G[:, k:] c with M_s[k:, k:] c = f[k:] (lower triangular)
            c = np.linalg.solve(np.tril(Ms[k:, k:]), f[k:])
            v = r - G[:, k:] @ c
            v = apply_M(v.reshape(shape)).ravel()
            U[:, k] = U[:, k:] @ c + omega * v
            G[:, k] = apply_A(U[:, k].reshape(shape)).ravel()
            info.iterations += 1
            for i in range(k):                  # G[:, k] perpendicular to P[:, :k]
                alpha = (P[:, i].conj() @ G[:, k]) / Ms[i, i]
                G[:, k] -= alpha * G[:, i]
                U[:, k] -= alpha * U[:, i]
            Ms[k:, k] = P[:, k:].conj().T @ G[:, k]
            if Ms[k, k] == 0:
                return xr.reshape(shape), info
            beta = f[k] / Ms[k, k]
            r = r - beta * G[:, k]
            xr = xr + beta * U[:, k]
            if _norm(r) <= tol * bnorm and accept():
                info.converged = True
                return xr.reshape(shape), info
            f[k + 1:] -= beta * Ms[k + 1:, k]
            if info.iterations >= maxit:
                break
        if info.iterations >= maxit:
            break
        # dimension reduction: r <- (I - omega A M^{-1}) r
        v = apply_M(r.reshape(shape)).ravel()
        t = apply_A(v.reshape(shape)).ravel()
        info.iterations += 1
        nt, nr, tr = _norm(t), _norm(r), complex(t.conj() @ r)
        omega = tr / nt ** 2
        rho = abs(tr) / (nt * nr) if nt > 0 and nr > 0 else 1.0
        if kappa > 0 and rho < kappa:
            omega = omega * kappa / rho
        xr = xr + omega * v
        r = r - omega * t
        info.history.append(_norm(r) / bnorm)
        if _norm(r) <= tol * bnorm and accept():
            info.converged = True
            return xr.reshape(shape), info
    info.rel_residual = _norm(b - apply_A(xr.reshape(shape))) / bnorm
    return xr.reshape(shape), info
