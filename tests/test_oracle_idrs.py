"""Pins of the oracle's IDR(s) (oracle.krylov.idrs; Sonneveld & van Gijzen 2008, biorthogonal
form of van Gijzen & Sonneveld 2011), a short-recurrence alternative to Bi-CGSTAB (Alg. 3) for the
strong-scattering workload (CPU):

* with s = 1, the shadow vector r_0 / ||r_0|| and the plain minimal-residual omega (kappa = 0) the
  method is Bi-CGSTAB: its residual after every dimension-reduction step equals the residual of
  oracle.krylov.bicgstab after every iteration (rounding apart), so a dropped term, a wrong sign
  or a missed biorthogonalisation step anywhere in the s = 1 path shows;
* for s = 2, 4, 8 (random orthonormal shadow space, kappa = 0.7) the iterate reaches the sparse
  direct solution of the same system;
* the reported residual is the true one, and a zero right-hand side returns zero at once;
* finite termination (the IDR theorem): on an n-dimensional system without preconditioning the
  residual vanishes after at most n + ceil(n / s) operator products, and not three products
  earlier, on small dense random systems.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.krylov import bicgstab, idrs


def _small(seed=5, n=24, levels=3):
    w = W.small_workload(n_int=n, abl=4, seed=seed, levels=levels)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    return p, f, O.MGHSolver(p, f, levels=levels, nu1=1, nu2=1, tol=1e-30)


def test_idr1_with_shadow_r0_is_bicgstab():
    p, f, s = _small()
    b = O.rhs(p, f, 0.4)
    r0 = (b - s.apply_A(np.zeros_like(b))).ravel()
    _, ib = bicgstab(s.apply_A, s.M, b, 1e-30, 40)
    _, ii = idrs(s.apply_A, s.M, b, 1e-30, 1, 40, shadow=r0[:, None] / np.linalg.norm(r0), kappa=0.0)
    assert ib.iterations == ii.iterations == 40
    hb, hi = np.array(ib.history), np.array(ii.history)
    assert len(hb) == len(hi) == 20
    # both fall by over two orders of magnitude; rounding drift grows slowly with the iteration count
    assert hb[-1] < 1e-2 * hb[0]
    np.testing.assert_allclose(hi[:8], hb[:8], rtol=1e-9)
    np.testing.assert_allclose(hi, hb, rtol=1e-4)


@pytest.mark.parametrize("sdim", [2, 4, 8])
def test_idrs_reaches_the_direct_solution(sdim):
    p, f, s = _small(seed=6)
    b = O.rhs(p, f, -0.7)
    x, info = idrs(s.apply_A, s.M, b, 1e-12, sdim, 600)
    assert info.converged
    ref = O.direct_solve(p, s.D, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    true_rel = np.linalg.norm(b - s.apply_A(x)) / np.linalg.norm(b)
    assert info.rel_residual == pytest.approx(true_rel, rel=1e-12)
    assert info.rel_residual <= 1e-12


def test_idrs_zero_rhs_and_iteration_cap():
    p, f, s = _small()
    b = O.rhs(p, f, 0.4)
    x, info = idrs(s.apply_A, s.M, np.zeros_like(b), 1e-8, 4, 50)
    assert info.converged and info.iterations == 0 and not np.any(x)
    _, info = idrs(s.apply_A, s.M, b, 1e-30, 4, 7)
    assert not info.converged and info.iterations == 7


@pytest.mark.parametrize("n,s", [(12, 4), (12, 3), (10, 2), (9, 1)])
def test_idrs_terminates_within_n_plus_n_over_s_products(n, s):
    rng = np.random.default_rng(10 * n + s)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    bound = n + -(-n // s)

    def run(maxit):
        x, info = idrs(lambda v: A @ v, lambda v: v, b, 1e-30, s, maxit, kappa=0.0, seed=3)
        assert info.iterations == maxit
        return np.linalg.norm(b - A @ x) / np.linalg.norm(b)

    assert run(bound) < 1e-8          # rounding level (cond(A) up to ~40)
    assert run(bound - 3) > 1e-5
