"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: the local Fourier symbols
of Sec. IV-B, exact discrete identities of the transfer operators (Sec. IV-C), a library LU
solve, a manufactured solution, the textbook multigrid iteration-matrix identity, finite
differences of the data term (Prop. 1), and the free-space Green's function.
"""
import math

import numpy as np
import pytest
import scipy.special as ssp

import oracle as O
import workloads as W


def plane_wave_grid(ny, nx, t1, t2):
    m = np.arange(nx)[None, :]
    n = np.arange(ny)[:, None]
    return np.exp(1j * (t1 * m + t2 * n))


def interior_mask(p, margin=1):
    """Points of Omega at least `margin` cells from the grid edge (alpha = 1 there)."""
    mask = np.zeros((p.ny, p.nx), dtype=bool)
    a = max(p.abl, margin)
    mask[a:p.ny - a, a:p.nx - a] = True
    return mask


THETAS = [(0.0, 0.0), (0.3, -1.1), (math.pi / 2, 0.7), (2.5, 3.0), (-math.pi, 1.3)]


@pytest.mark.parametrize("t1,t2", THETAS)
def test_stencil_matches_lfa_symbol(t1, t2):
    """Interior rows of A act on e^{j(t1 m + t2 n)} as a^h(theta) = (4 - 2cos t1 - 2cos t2 - k^2h^2)/h^2 (Sec. IV-B)."""
    p = O.Problem(20, 14, 5, h=0.37, k=2 * math.pi / 7.0, beta=0.3)
    c = O.fine_coefficient(p, np.zeros((p.ny_int, p.nx_int)))
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    v = plane_wave_grid(p.ny, p.nx, t1, t2)
    Av = O.apply_operator(D, v, p.h)
    a_h = (4 - 2 * math.cos(t1) - 2 * math.cos(t2) - p.k ** 2 * p.h ** 2) / p.h ** 2
    mask = interior_mask(p)
    np.testing.assert_allclose(Av[mask], a_h * v[mask], rtol=0, atol=1e-12 * (8 / p.h ** 2))


@pytest.mark.parametrize("t1,t2", THETAS)
def test_shifted_operator_symbol(t1, t2):
    """K_kappa = -lap - kappa k^2 has symbol (4 - 2cos t1 - 2cos t2)/h^2 - kappa k^2 on Omega (Sec. IV-B)."""
    p = O.Problem(18, 18, 4, h=1.0, k=2 * math.pi / 10.0)
    c = O.fine_coefficient(p, np.zeros((p.ny_int, p.nx_int)))
    kappa = 1 + 0.5j
    hier = O.build_hierarchy(p, c, 1, kappa)
    v = plane_wave_grid(p.ny, p.nx, t1, t2)
    Kv = O.apply_operator(hier[0].D, v, p.h)
    sym = (4 - 2 * math.cos(t1) - 2 * math.cos(t2)) / p.h ** 2 - kappa * p.k ** 2
    mask = interior_mask(p)
    np.testing.assert_allclose(Kv[mask], sym * v[mask], rtol=0, atol=1e-12)


@pytest.mark.parametrize("t1,t2", THETAS)
def test_jacobi_symbol(t1, t2):
    """One damped Jacobi step on the error e^{j theta.x} multiplies it by
    s^h(theta) = 1 - w + 2w (cos t1 + cos t2)/(4 - k^2 h^2) (Sec. IV-B, unshifted, constant k)."""
    p = O.Problem(16, 16, 4, h=1.0, k=2 * math.pi / 10.0)
    c = O.fine_coefficient(p, np.zeros((p.ny_int, p.nx_int)))
    lv = O.build_hierarchy(p, c, 1, 1.0)[0]
    w = 0.8
    e = plane_wave_grid(p.ny, p.nx, t1, t2)
    e1 = O.jacobi(lv, np.zeros_like(e), e, w)
    s = 1 - w + 2 * w * (math.cos(t1) + math.cos(t2)) / (4 - (p.k * p.h) ** 2)
    mask = interior_mask(p)
    np.testing.assert_allclose(e1[mask], s * e[mask], rtol=0, atol=1e-13)


def test_jacobi_divergence_bound():
    """max_theta |s^h| = 1 - w + 4w/(4 - k^2h^2) > 1 (Sec. IV-B), reached by the smooth mode."""
    p = O.Problem(16, 16, 4, h=1.0, k=2 * math.pi / 10.0)
    c = O.fine_coefficient(p, np.zeros((p.ny_int, p.nx_int)))
    lv = O.build_hierarchy(p, c, 1, 1.0)[0]
    w = 0.8
    mask = interior_mask(p)
    best = 0.0
    for t1 in np.linspace(-math.pi, math.pi, 13):
        for t2 in np.linspace(-math.pi, math.pi, 13):
            e = plane_wave_grid(p.ny, p.nx, t1, t2)
            e1 = O.jacobi(lv, np.zeros_like(e), e, w)
            best = max(best, float(np.max(np.abs(e1[mask] / e[mask]))))
    bound = 1 - w + 4 * w / (4 - (p.k * p.h) ** 2)
    assert bound > 1.0
    assert abs(best - bound) < 1e-12


@pytest.mark.parametrize("ny,nx", [(7, 9), (8, 8), (10, 13), (12, 6), (3, 3), (2, 5)])
def test_restriction_prolongation_adjoint_exact(ny, nx):
    """P is the adjoint of R with the 1/16 weights: 4 <R x, y> = <x, P y>, bit-exact on integers (Sec. IV-C)."""
    rng = np.random.default_rng(ny * 100 + nx)
    x = rng.integers(-50, 50, size=(ny, nx)).astype(np.float64)
    y = rng.integers(-50, 50, size=(O.coarse_size(ny), O.coarse_size(nx))).astype(np.float64)
    lhs = 4.0 * np.sum(O.restrict(x) * y)
    rhs = np.sum(x * O.prolong(y, ny, nx))
    assert lhs == rhs


def _restrict_brute(r):
    ny, nx = r.shape
    nyc, nxc = O.coarse_size(ny), O.coarse_size(nx)
    out = np.zeros((nyc, nxc), dtype=r.dtype)

    def at(n, m):
        return r[n, m] if (0 <= n < ny and 0 <= m < nx) else 0.0

    for j in range(nyc):
        for i in range(nxc):
            m, n = 2 * i, 2 * j
            out[j, i] = (4 * at(n, m)
                         + 2 * (at(n, m - 1) + at(n, m + 1) + at(n - 1, m) + at(n + 1, m))
                         + at(n - 1, m - 1) + at(n + 1, m - 1) + at(n - 1, m + 1) + at(n + 1, m + 1)) / 16.0
    return out


def _prolong_brute(ec, ny, nx):
    nyc, nxc = ec.shape

    def at(j, i):
        return ec[j, i] if (0 <= j < nyc and 0 <= i < nxc) else 0.0

    e = np.zeros((ny, nx), dtype=ec.dtype)
    for n in range(ny):
        for m in range(nx):
            if m % 2 == 0 and n % 2 == 0:
                e[n, m] = at(n // 2, m // 2)
            elif m % 2 == 1 and n % 2 == 0:
                e[n, m] = 0.5 * (at(n // 2, (m - 1) // 2) + at(n // 2, (m + 1) // 2))
            elif m % 2 == 0 and n % 2 == 1:
                e[n, m] = 0.5 * (at((n - 1) // 2, m // 2) + at((n + 1) // 2, m // 2))
            else:
                e[n, m] = 0.25 * (at((n - 1) // 2, (m - 1) // 2) + at((n + 1) // 2, (m - 1) // 2)
                                  + at((n - 1) // 2, (m + 1) // 2) + at((n + 1) // 2, (m + 1) // 2))
    return e


@pytest.mark.parametrize("ny,nx", [(7, 9), (8, 8), (11, 6), (1, 4)])
def test_transfer_operators_brute_force(ny, nx):
    rng = np.random.default_rng(3)
    r = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    np.testing.assert_allclose(O.restrict(r), _restrict_brute(r), rtol=0, atol=1e-15)
    ec = rng.standard_normal((O.coarse_size(ny), O.coarse_size(nx)))
    np.testing.assert_allclose(O.prolong(ec, ny, nx), _prolong_brute(ec, ny, nx), rtol=0, atol=1e-15)


def test_restriction_keeps_constants_and_prolongation_keeps_bilinear():
    ny, nx = 13, 16
    rc = O.restrict(np.ones((ny, nx)))
    assert np.all(rc[1:-1, 1:-1] == 1.0)
    nyc, nxc = O.coarse_size(ny), O.coarse_size(nx)
    I, J = np.meshgrid(np.arange(nxc), np.arange(nyc))
    ec = 3.0 + 2.0 * (2 * I) - 5.0 * (2 * J) + 0.25 * (2 * I) * (2 * J)   # bilinear in fine coords
    e = O.prolong(ec, ny, nx)
    M, N = np.meshgrid(np.arange(nx), np.arange(ny))
    ref = 3.0 + 2.0 * M - 5.0 * N + 0.25 * M * N
    inside = (M <= 2 * (nxc - 1)) & (N <= 2 * (nyc - 1))
    np.testing.assert_array_equal(e[inside], ref[inside])


def test_prolongation_is_four_times_restriction_transpose():
    ny, nx = 9, 8
    nyc, nxc = O.coarse_size(ny), O.coarse_size(nx)
    R = np.zeros((nyc * nxc, ny * nx))
    for q in range(ny * nx):
        u = np.zeros(ny * nx)
        u[q] = 1.0
        R[:, q] = O.restrict(u.reshape(ny, nx)).ravel()
    P = np.zeros((ny * nx, nyc * nxc))
    for q in range(nyc * nxc):
        u = np.zeros(nyc * nxc)
        u[q] = 1.0
        P[:, q] = O.prolong(u.reshape(nyc, nxc), ny, nx).ravel()
    np.testing.assert_array_equal(P, 4.0 * R.T)


def _small(nint=16, abl=4, seed=5, beta=0.15, ppw=8.0):
    p = O.Problem(nint, nint + 2, abl, h=1.0, k=2 * math.pi / ppw, beta=beta)
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.0, 0.4, size=(p.ny_int, p.nx_int))
    return p, f


def test_operator_complex_symmetric_and_absorbing():
    """A^T = A exactly, Im diag(A) <= 0 (absorbing reading), matrix-free apply = sparse matvec."""
    p, f = _small()
    c = O.fine_coefficient(p, f)
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    A = O.assemble_operator(D, p.h)
    assert (A - A.T).count_nonzero() == 0
    assert np.all(D.imag <= 0.0)
    assert np.all(D.imag[0, :] < 0.0) and np.all(D.imag[:, -1] < 0.0)
    x = W.random_field((p.ny, p.nx), 1)
    np.testing.assert_allclose(O.apply_operator(D, x, p.h).ravel(), A @ x.ravel(), rtol=1e-14, atol=1e-14)
    y = W.random_field((p.ny, p.nx), 2)
    lhs = np.vdot(y.ravel(), (A @ x.ravel()))
    rhs_ = np.vdot((A.conj().T @ y.ravel()), x.ravel())
    assert abs(lhs - rhs_) <= 1e-13 * abs(lhs)


def test_layout_x_is_fast_axis():
    """u_{m,n} is entry n*nx + m with x = m h (Sec. IV-A): a plane wave along +x varies along columns."""
    p = O.Problem(6, 4, 2, h=0.5, k=1.3)
    u = O.incident_field(p, 0.0)
    assert u.shape == (p.ny, p.nx)
    np.testing.assert_allclose(u[0, :], np.exp(1j * p.k * p.h * np.arange(p.nx)))
    np.testing.assert_array_equal(u, np.repeat(u[:1, :], p.ny, axis=0))


def test_layer_factor_geometry():
    """alpha = 1 on Omega, 1 + j beta at the outer edge of the layer along an axis, corners further."""
    p = O.Problem(10, 8, 3, h=1.0, k=1.0, beta=0.2)
    a = O.absorbing_factor(p)
    assert np.all(a[3:11, 3:13] == 1.0)
    assert a[5, 0] == pytest.approx(1 + 0.2j, abs=1e-15) and a[0, 7] == pytest.approx(1 + 0.2j, abs=1e-15)
    assert a[0, 0] == pytest.approx(1 + 0.4j, abs=1e-15)
    assert a[5, 1] == pytest.approx(1 + 0.2j * 4 / 9, abs=1e-15)


def test_level_counts():
    sizes = {160: [160, 80, 40, 20], 576: [576, 288, 144, 72, 36, 18], 1120: [1120, 560, 280, 140, 70, 35]}
    for n, ref in sizes.items():
        out = [n]
        while len(out) < len(ref):
            out.append(O.coarse_size(out[-1]))
        assert out == ref


def test_gmres_matches_direct_solve():
    """FGMRES to rel. residual 1e-13 agrees with a sparse LU solve (SuperLU) within 1e-10."""
    p, f = _small()
    s = O.MGHSolver(p, f, levels=3, nu1=1, nu2=1, restart=20, tol=1e-13)
    b = O.rhs(p, f, 0.4)
    u, info = s.solve(b)
    assert info.converged
    ref = O.direct_solve(p, s.D, b)
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("m", [1, 4, 8])
def test_sstep_cycle_equals_arnoldi_cycle(m):
    """One s-step cycle (Gram matrix + Cholesky) returns the iterate of one Arnoldi cycle of
    FGMRES(m) from the same starting point: both minimise the residual over x + span(Z), with the
    same z_k because the preconditioner sees the same normalised vectors."""
    from oracle.krylov import fgmres, sstep_cycle
    p, f = _small(seed=5)
    s = O.MGHSolver(p, f, levels=3, nu1=1, nu2=1, restart=m, tol=1e-30)
    b = O.rhs(p, f, 0.2)
    x0 = W.random_field((p.ny, p.nx), 3) * 1e-2
    x_ar, info = fgmres(s.apply_A, s.M, b, 1e-30, m, m, x0)
    assert info.iterations == m
    x_ss = sstep_cycle(s.apply_A, s.M, b, x0, m)
    assert np.linalg.norm(x_ss - x_ar) <= 1e-9 * np.linalg.norm(x_ar)
    # and the cycle reduced the residual
    r0 = np.linalg.norm(b - s.apply_A(x0))
    assert np.linalg.norm(b - s.apply_A(x_ss)) < r0


def _gram_fp32_runs(Vm, run=32, lanes=64):
    """The Gram matrix as the CUDA s-step sweep forms it: the basis stored in FP32, every product
    of a pair rounded to FP32 and summed in FP32 in runs of `run` products per lane (a lane takes
    every `lanes`-th point), the run sums added exactly (here in FP64)."""
    V = Vm.astype(np.complex64)
    N, nv = V.shape
    per = run * lanes
    pad = (-N) % per
    G = np.zeros((nv, nv), dtype=np.complex128)
    for i in range(nv):
        for j in range(i, nv):
            P = np.conj(V[:, i]) * V[:, j]
            P = np.concatenate([P, np.zeros(pad, np.complex64)]).reshape(-1, run, lanes)
            s = P[:, 0, :].copy()
            for t in range(1, run):
                s = (s + P[:, t, :]).astype(np.complex64)
            G[i, j] = s.astype(np.complex128).sum()
            G[j, i] = np.conj(G[i, j])
    return G


def test_sstep_cycles_need_only_fp32_gram_sums():
    """The reading behind the CUDA Gram sweep's FP32 running sums: s-step FGMRES(8) cycles whose
    Gram matrix is that of the FP32-rounded basis summed in FP32 runs of 32 products take the same
    steps to 1e-8 as cycles with the exact FP64 Gram matrix, and reach the same residual.  The
    rounded Gram stays within the recursive-summation bound (run + 1) u32 sum_p |v_i[p]| |v_j[p]|
    of the Gram of the rounded basis, so its error is a normwise perturbation of size
    FP32 storage of the basis already makes."""
    from oracle.krylov import sstep_cycle
    w = W.Workload("sstep96", 96, 96, 12, 10.0, 1, 0.0, 0.0, "ellipses", 2, levels=4, nu1=2, nu2=2, restart=8)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    s = O.MGHSolver(p, f, levels=4, nu1=2, nu2=2, restart=8, tol=1e-8)
    b = O.rhs(p, f, 0.3)
    nb = np.linalg.norm(b)
    out = {}
    for name, gram in (("fp64", None), ("fp32_runs", _gram_fp32_runs)):
        x = np.zeros_like(b)
        steps = 0
        while np.linalg.norm(b - s.apply_A(x)) > 1e-8 * nb and steps < 2000:
            x = sstep_cycle(s.apply_A, s.M, b, x, 8, gram=gram)
            steps += 8
        out[name] = (steps, np.linalg.norm(b - s.apply_A(x)) / nb)
    assert out["fp64"][0] < 2000 and out["fp32_runs"][0] == out["fp64"][0], out
    assert out["fp32_runs"][1] <= 1e-8 and abs(out["fp32_runs"][1] - out["fp64"][1]) <= 1e-2 * out["fp64"][1]
    # the error model on a basis of this problem (the V-cycle's monomial basis of one cycle)
    r = b.copy()
    Vs = [r / np.linalg.norm(r)]
    for _ in range(8):
        wv = s.apply_A(s.M(Vs[-1]))
        Vs.append(wv / np.linalg.norm(wv))
    Vm = np.stack([v.ravel() for v in Vs], axis=1)
    V32 = Vm.astype(np.complex64).astype(np.complex128)
    G_ref = V32.conj().T @ V32
    bound = 33 * np.finfo(np.float32).eps * (np.abs(V32).T @ np.abs(V32)) * 2
    err = np.abs(_gram_fp32_runs(Vm) - G_ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_bicgstab_matches_direct_solve():
    p, f = _small(seed=9)
    s = O.MGHSolver(p, f, levels=2, nu1=1, nu2=1, tol=1e-12, krylov="bicgstab", shift=1.0)
    b = O.rhs(p, f, -0.7)
    u, info = s.solve(b)
    assert info.converged
    ref = O.direct_solve(p, s.D, b)
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)


def test_manufactured_solution():
    p, f = _small(seed=11)
    s = O.MGHSolver(p, f, levels=3, nu1=2, nu2=2, tol=1e-13)
    X, Y = np.meshgrid(np.arange(p.nx), np.arange(p.ny))
    u_star = np.sin(0.3 * X) * np.cos(0.2 * Y) * np.exp(-((X - 12) ** 2 + (Y - 13) ** 2) / 60.0) * (1 + 0.5j)
    A = O.assemble_operator(s.D, p.h)
    b = (A @ u_star.ravel()).reshape(u_star.shape)
    u, info = s.solve(b)
    assert info.converged
    assert np.linalg.norm(u - u_star) <= 1e-10 * np.linalg.norm(u_star)


def test_zero_contrast_gives_zero_field():
    p = O.Problem(12, 12, 3, h=1.0, k=0.7)
    f = np.zeros((12, 12))
    s = O.MGHSolver(p, f, levels=2, nu1=1, nu2=1)
    u, infos = s.forward([0.0, 1.0])
    assert np.all(u == 0.0)
    assert all(i.iterations == 0 and i.converged for i in infos)


def _dense(op, n):
    M = np.zeros((n, n), dtype=np.complex128)
    for q in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[q] = 1.0
        M[:, q] = op(e)
    return M


def _vcycle_matrix_closed_form(hier, l, nu1, nu2, omega):
    """Textbook MG identity (zero initial guess): M_l^{-1} = (I - E_l) K_l^{-1},
    E_l = S^nu2 (I - P M_{l+1}^{-1} R K_l) S^nu1, S = I - omega D^{-1} K_l; coarsest M^{-1} = K^{-1}."""
    lv = hier[l]
    n = lv.nx * lv.ny
    K = O.assemble_operator(lv.D, lv.h).toarray()
    Kinv = np.linalg.inv(K)
    if l == len(hier) - 1:
        return Kinv
    c = hier[l + 1]
    nc = c.nx * c.ny
    R = _dense(lambda e: O.restrict(e.reshape(lv.ny, lv.nx)).ravel(), n)[:nc, :] if False else \
        np.stack([O.restrict(np.eye(n)[q].reshape(lv.ny, lv.nx)).ravel() for q in range(n)], axis=1)
    P = np.stack([O.prolong(np.eye(nc)[q].reshape(c.ny, c.nx), lv.ny, lv.nx).ravel() for q in range(nc)], axis=1)
    S = np.eye(n) - omega * np.diag(1.0 / lv.D.ravel()) @ K
    Mc = _vcycle_matrix_closed_form(hier, l + 1, nu1, nu2, omega)
    E = np.linalg.matrix_power(S, nu2) @ (np.eye(n) - P @ Mc @ R @ K) @ np.linalg.matrix_power(S, nu1)
    return (np.eye(n) - E) @ Kinv


@pytest.mark.parametrize("nu", [0, 1, 2])
def test_vcycle_equals_iteration_matrix_identity(nu):
    p = O.Problem(8, 6, 2, h=1.0, k=2 * math.pi / 6.0, beta=0.3)
    rng = np.random.default_rng(4)
    f = rng.uniform(0, 0.3, size=(p.ny_int, p.nx_int))
    c = O.fine_coefficient(p, f)
    pre = O.Preconditioner(p, c, levels=3, nu1=nu, nu2=nu, omega=0.8, shift=1 + 0.5j)
    n = p.nx * p.ny
    M_proc = _dense(lambda e: pre(e.reshape(p.ny, p.nx)).ravel(), n)
    M_ref = _vcycle_matrix_closed_form(pre.hier, 0, nu, nu, 0.8)
    assert np.max(np.abs(M_proc - M_ref)) <= 1e-11 * np.max(np.abs(M_ref))


def _gamma_cycle_matrix(hier, l, nu1, nu2, omega, gamma):
    """Textbook identity of the gamma-cycle with per-level sweeps (Trottenberg et al. 2000, Sec.
    2.4): M_l^{-1} = (I - E_l) K_l^{-1}, E_l = S_l^{nu2_l} (I - P Mg_{l+1} R K_l) S_l^{nu1_l}, where
    Mg_{l+1} = (I - (I - M_{l+1}^{-1} K_{l+1})^gamma) K_{l+1}^{-1} is gamma cycles of level l + 1
    from a zero guess; on the coarsest level M^{-1} = K^{-1}.  Built from dense matrices only."""
    lv = hier[l]
    n = lv.nx * lv.ny
    K = O.assemble_operator(lv.D, lv.h).toarray()
    Kinv = np.linalg.inv(K)
    if l == len(hier) - 1:
        return Kinv
    c = hier[l + 1]
    nc = c.nx * c.ny
    Kc = O.assemble_operator(c.D, c.h).toarray()
    R = np.stack([O.restrict(np.eye(n)[q].reshape(lv.ny, lv.nx)).ravel() for q in range(n)], axis=1)
    P = np.stack([O.prolong(np.eye(nc)[q].reshape(c.ny, c.nx), lv.ny, lv.nx).ravel() for q in range(nc)], axis=1)
    S = np.eye(n) - omega * np.diag(1.0 / lv.D.ravel()) @ K
    Mc = _gamma_cycle_matrix(hier, l + 1, nu1, nu2, omega, gamma)
    Ec = np.eye(nc) - Mc @ Kc
    Mg = (np.eye(nc) - np.linalg.matrix_power(Ec, gamma)) @ np.linalg.inv(Kc)
    E = np.linalg.matrix_power(S, nu2[l]) @ (np.eye(n) - P @ Mg @ R @ K) @ np.linalg.matrix_power(S, nu1[l])
    return (np.eye(n) - E) @ Kinv


@pytest.mark.parametrize("gamma,nu1,nu2", [(2, (1, 1, 1), (1, 1, 1)), (2, (2, 0, 1), (0, 1, 2)),
                                           (3, (1, 2, 1), (2, 1, 0)), (1, (0, 2, 1), (1, 0, 2))])
def test_w_cycle_and_per_level_sweeps_equal_iteration_matrix_identity(gamma, nu1, nu2):
    p = O.Problem(14, 10, 2, h=1.0, k=2 * math.pi / 6.0, beta=0.3)
    rng = np.random.default_rng(9)
    f = rng.uniform(0, 0.3, size=(p.ny_int, p.nx_int))
    c = O.fine_coefficient(p, f)
    pre = O.Preconditioner(p, c, levels=4, nu1=list(nu1) + [0], nu2=list(nu2) + [0], omega=0.8,
                           shift=1 + 0.5j, cycle_type=gamma)
    n = p.nx * p.ny
    M_proc = _dense(lambda e: pre(e.reshape(p.ny, p.nx)).ravel(), n)
    M_ref = _gamma_cycle_matrix(pre.hier, 0, list(nu1) + [0], list(nu2) + [0], 0.8, gamma)
    assert np.max(np.abs(M_proc - M_ref)) <= 1e-10 * np.max(np.abs(M_ref))


@pytest.mark.parametrize("gamma,levels", [(1, 4), (2, 4), (2, 5), (3, 4)])
def test_cycle_type_visits_the_coarsest_level_gamma_to_the_depth(gamma, levels):
    """Alg. 2 with CycleType = gamma calls the coarsest solve gamma^(L-1) times: every level
    0..L-2 calls the next one gamma times."""
    p = O.Problem(30, 30, 2, h=1.0, k=0.9)
    c = O.fine_coefficient(p, np.full((30, 30), 0.1))
    pre = O.Preconditioner(p, c, levels=levels, nu1=1, nu2=1, omega=0.8, shift=1 + 0.5j, cycle_type=gamma)
    calls = []
    inner = pre.coarse
    pre.coarse = lambda b: (calls.append(1), inner(b))[1]
    pre(W.random_field((p.ny, p.nx), 2))
    assert len(calls) == gamma ** (levels - 1)


def test_w_cycle_on_two_levels_is_the_two_grid_cycle():
    """With an exact coarse solve, repeating it changes nothing: CycleType 2 on two levels is
    Alg. 1 (the two-grid cycle)."""
    p = O.Problem(12, 10, 2, h=1.0, k=0.9)
    c = O.fine_coefficient(p, np.full((10, 12), 0.2))
    b = W.random_field((p.ny, p.nx), 5)
    v = O.Preconditioner(p, c, levels=2, nu1=2, nu2=1, omega=0.8, shift=1 + 0.5j, cycle_type=1)(b)
    w = O.Preconditioner(p, c, levels=2, nu1=2, nu2=1, omega=0.8, shift=1 + 0.5j, cycle_type=2)(b)
    np.testing.assert_allclose(w, v, rtol=0, atol=1e-13 * np.abs(v).max())


def test_two_grid_without_smoothing_is_p_kinv_r():
    """Alg. 1 with nu1 = nu2 = 0 and an exact coarse solve is P K_c^{-1} R."""
    p = O.Problem(10, 10, 2, h=1.0, k=0.9)
    c = O.fine_coefficient(p, np.full((10, 10), 0.2))
    pre = O.Preconditioner(p, c, levels=2, nu1=0, nu2=0, omega=0.8, shift=1 + 0.5j)
    b = W.random_field((p.ny, p.nx), 3)
    cl = pre.hier[1]
    Kc = O.assemble_operator(cl.D, cl.h).toarray()
    ref = O.prolong(np.linalg.solve(Kc, O.restrict(b).ravel()).reshape(cl.ny, cl.nx), p.ny, p.nx)
    np.testing.assert_allclose(pre(b), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_coarse_coefficient_ring_is_background():
    p = O.Problem(20, 20, 4, h=1.0, k=0.8)
    f = np.full((20, 20), 0.5)
    c = O.fine_coefficient(p, f)
    hier = O.build_hierarchy(p, c, 3, 1.0)
    for lv in hier[1:]:
        assert np.all(lv.c[0, :] == p.k ** 2) and np.all(lv.c[:, -1] == p.k ** 2)
    # interior coarse points average the fine coefficient (full weighting of a constant)
    assert hier[1].c[8, 8] == pytest.approx(p.k ** 2 * 1.5)


def _fd_problem():
    p = O.Problem(10, 10, 3, h=1.0, k=2 * math.pi / 6.0, beta=0.3)
    rng = np.random.default_rng(21)
    f = rng.uniform(0.0, 0.3, size=(10, 10))
    thetas = [0.0, 0.6]
    rec = np.array([(p.abl + n) * p.nx + p.abl + 8 for n in range(p.ny_int)], dtype=np.int64)
    y = W.random_field((2, rec.size), 22) * 0.1
    return p, f, thetas, rec, y


def _loss_direct(p, f, thetas, rec, y):
    c = O.fine_coefficient(p, f)
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    us = np.stack([O.direct_solve(p, D, O.rhs(p, f, t)) for t in thetas])
    return O.misfit(O.sample(us, rec), y)[1]


def test_gradient_matches_finite_differences():
    """dL/df_d from one adjoint solve per angle (Prop. 1) vs central differences of L."""
    p, f, thetas, rec, y = _fd_problem()
    s = O.MGHSolver(p, f, levels=2, nu1=1, nu2=1, tol=1e-13)
    loss, g, _ = s.gradient(thetas, rec, y)
    assert loss == pytest.approx(_loss_direct(p, f, thetas, rec, y), rel=1e-10)
    rng = np.random.default_rng(5)
    for _ in range(4):
        d = rng.standard_normal(f.shape)
        eps = 1e-5
        fd = (_loss_direct(p, f + eps * d, thetas, rec, y) - _loss_direct(p, f - eps * d, thetas, rec, y)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_prop1_linearisation():
    """d u_sc = A^{-1} diag(u) k^2 df_d (Prop. 1) vs central differences of the solution."""
    p, f, thetas, _, _ = _fd_problem()
    rng = np.random.default_rng(8)
    v = rng.standard_normal(f.shape)
    c = O.fine_coefficient(p, f)
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    u_sc = O.direct_solve(p, D, O.rhs(p, f, 0.3))
    u = u_sc + O.incident_field(p, 0.3)
    jv = O.direct_solve(p, D, p.k ** 2 * O.embed(p, v) * u)
    eps = 1e-6

    def usc(ff):
        cc = O.fine_coefficient(p, ff)
        DD = O.operator_diagonal(cc, O.absorbing_factor(p), p.h, p.k)
        return O.direct_solve(p, DD, O.rhs(p, ff, 0.3))

    fd = (usc(f + eps * v) - usc(f - eps * v)) / (2 * eps)
    assert np.linalg.norm(jv - fd) <= 1e-7 * np.linalg.norm(jv)


def test_point_source_is_outgoing():
    """With the damping sign reading, a point source radiates like (j/4) H0^(1)(k r), the outgoing
    free-space Green's function of -lap - k^2 under the e^{-j w t} convention (Sec. II-A)."""
    p = O.Problem(60, 60, 30, h=1.0, k=2 * math.pi / 12.0, beta=1.0)
    c = O.fine_coefficient(p, np.zeros((60, 60)))
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    b = np.zeros((p.ny, p.nx), dtype=np.complex128)
    cy = cx = p.abl + 30
    b[cy, cx] = 1.0 / p.h ** 2
    u = O.direct_solve(p, D, b)
    X, Y = np.meshgrid(np.arange(p.nx), np.arange(p.ny))
    r = np.hypot(X - cx, Y - cy) * p.h
    ring = (r > 8) & (r < 25)
    g_out = 0.25j * ssp.hankel1(0, p.k * r[ring])
    g_in = -0.25j * ssp.hankel2(0, p.k * r[ring])
    err_out = np.linalg.norm(u[ring] - g_out) / np.linalg.norm(g_out)
    err_in = np.linalg.norm(u[ring] - g_in) / np.linalg.norm(g_in)
    assert err_out < 0.1
    assert err_in > 1.0


def test_flexible_gmres_tolerates_fp16_rounded_preconditioned_vectors():
    """Flexible GMRES builds x from the stored preconditioned vectors z_j and their products A z_j,
    so rounding z_j (as FP16 storage would) changes the preconditioner, not the result: FGMRES(8)
    with the MG cycle's output rounded to half precision reaches the direct solution to the same
    tolerance in the same number of steps (within 2 %) as with the exact cycle."""
    w = W.Workload("r", 70, 53, 9, 8.0, 1, 0, 0, "ellipses", 11, levels=4, nu1=2, nu2=2, restart=8, tol=1e-10)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    s = O.MGHSolver(p, f, 4, 2, 2, 0.8, 1 + 0.5j, 8, 1e-10, maxit=3000)
    b = O.rhs(p, f, 0.3)
    ref = O.direct_solve(p, s.D, b)
    half = lambda z: z.real.astype(np.float16).astype(np.float64) + 1j * z.imag.astype(np.float16).astype(np.float64)
    x0, i0 = O.fgmres(s.apply_A, s.M, b, 1e-10, 8, 3000)
    x1, i1 = O.fgmres(s.apply_A, lambda r: half(s.M(r)), b, 1e-10, 8, 3000)
    assert i0.converged and i1.converged
    assert abs(i1.iterations - i0.iterations) <= 0.02 * i0.iterations + 1
    for x in (x0, x1):
        assert np.linalg.norm(b - s.apply_A(x)) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-9)
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
