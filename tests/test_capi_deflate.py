"""The host routine of the deflated restart (mgh_debug_deflate, the code the solver runs between
cycles) against the oracle's harmonic Ritz problem and restart (CPU only: no device work).

The routine returns C = P_k W (the k harmonic Ritz vectors of smallest modulus, orthonormalised,
times a unitary W), the Arnoldi matrix Hh of the kept columns in upper Hessenberg form and its
Givens QR.  Pins: C spans the oracle's harmonic Ritz vectors; Hbar C = [[C; 0], c~] Hh with c~ the
residual coefficients orthogonalised against C (the relation A Z' = V' Hh the next cycle extends);
Hh is Hessenberg and the rotations reduce it to the returned triangle; the kept basis and Hh are
the oracle's deflated_restart up to that unitary change of basis."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.krylov import deflated_restart, harmonic_ritz


@pytest.fixture(scope="module")
def capi():
    import os
    from paper_2107_03679_gb300 import build
    if not os.path.exists(build.LIB):
        import __graft_entry__ as g
        g.build()
    from paper_2107_03679_gb300 import capi as c
    return c


def _arnoldi_matrix(seed, m):
    """Hbar of m Arnoldi steps of the multigrid-preconditioned operator of a small workload."""
    w = W.small_workload(n_int=20, abl=4, seed=seed, levels=3)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    s = O.MGHSolver(p, f, levels=3, nu1=1, nu2=1, tol=1e-30)
    b = O.rhs(p, f, 0.1 * seed)
    n = b.size
    V = np.zeros((n, m + 1), complex)
    H = np.zeros((m + 1, m), complex)
    beta = np.linalg.norm(b)
    V[:, 0] = b.ravel() / beta
    for j in range(m):
        w_ = s.apply_A(s.M(V[:, j].reshape(b.shape))).ravel()
        for _ in range(2):
            h = V[:, :j + 1].conj().T @ w_
            w_ -= V[:, :j + 1] @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w_)
        V[:, j + 1] = w_ / H[j + 1, j]
    return H, beta


def _span_gap(A, B):
    """Largest distance of a unit column of B from range(A) (A with orthonormal columns)."""
    Bn = B / np.linalg.norm(B, axis=0)
    return float(np.max(np.linalg.norm(Bn - A @ (A.conj().T @ Bn), axis=0)))


def _residual_coefficients(H, beta):
    m = H.shape[1]
    g = np.zeros(m + 1, complex)
    g[0] = beta
    y = np.linalg.lstsq(H, g, rcond=None)[0]
    return g - H @ y


@pytest.mark.parametrize("seed,m,k", [(1, 8, 4), (2, 12, 6), (3, 20, 10), (4, 16, 1), (5, 32, 16)])
def test_host_restart_data_matches_the_harmonic_ritz_problem(capi, seed, m, k):
    H, beta = _arnoldi_matrix(seed, m)
    c = _residual_coefficients(H, beta)
    C, Hh, R, cs, sn = capi.mgh_debug_deflate(H, c, k)
    # orthonormal C spanning the oracle's k harmonic Ritz vectors, an invariant subspace of T
    assert np.linalg.norm(C.conj().T @ C - np.eye(k)) <= 1e-12
    assert _span_gap(C, harmonic_ritz(H, k)) <= 1e-8
    Hm = H[:m, :]
    e = np.zeros(m)
    e[-1] = 1.0
    T = Hm + abs(H[m, m - 1]) ** 2 * np.outer(np.linalg.solve(Hm.conj().T, e), e)
    TC = T @ C
    assert np.linalg.norm(TC - C @ (C.conj().T @ TC)) <= 1e-8 * np.linalg.norm(TC)
    # the kept relation: Hbar C = [[C; 0], c~] Hh, c~ the residual direction orthogonal to C
    Cp = np.vstack([C, np.zeros((1, k))])
    ct = c - Cp @ (Cp.conj().T @ c)
    ct /= np.linalg.norm(ct)
    Vn = np.hstack([Cp, ct[:, None]])
    assert np.linalg.norm(H @ C - Vn @ Hh) <= 1e-9 * np.linalg.norm(H @ C)
    assert np.linalg.norm(c - Vn @ (Vn.conj().T @ c)) <= 1e-9 * np.linalg.norm(c)   # r stays in span(V')
    # Hessenberg form and its Givens QR
    assert np.all(Hh[np.tril_indices(k + 1, -2, k)] == 0)
    Rr = Hh.copy()
    for i in range(k):
        a, b = Rr[i].copy(), Rr[i + 1].copy()
        Rr[i], Rr[i + 1] = cs[i] * a + sn[i] * b, -np.conj(sn[i]) * a + cs[i] * b
    assert np.linalg.norm(Rr[:k] - R) <= 1e-12 * np.linalg.norm(R)
    assert np.linalg.norm(Rr[k]) <= 1e-12 * np.linalg.norm(R) and np.allclose(np.tril(R, -1), 0.0)
    # the oracle's restart: same kept basis and Arnoldi matrix up to a unitary change of basis
    Vo, _, Ho, go = deflated_restart(np.eye(m + 1), np.eye(m + 1)[:m, :m], H, c, k)
    U = Vo.conj().T @ Vn                  # (k+1) x (k+1), unitary when the spans agree
    assert np.linalg.norm(U.conj().T @ U - np.eye(k + 1)) <= 1e-8
    assert np.linalg.norm(Hh - U.conj().T @ Ho @ U[:k, :k]) <= 1e-8 * np.linalg.norm(Hh)


def test_arguments_are_checked(capi):
    H, beta = _arnoldi_matrix(1, 8)
    c = _residual_coefficients(H, beta)
    for k in (0, 8):
        with pytest.raises(capi.MGHError) as e:
            capi.mgh_debug_deflate(H, c, k)
        assert e.value.status == capi.MGH_INVALID_ARG


def test_deflate_parameter_validation(capi):
    p = capi.mgh_default_params()
    p.deflate = 10
    base = capi.mgh_workspace_bytes(capi.mgh_default_params())
    assert capi.mgh_workspace_bytes(p) > base                 # raw Hessenberg and restart data
    for restart, k, status in ((20, 20, capi.MGH_INVALID_ARG), (20, 17, capi.MGH_INVALID_ARG),
                               (20, -1, capi.MGH_INVALID_ARG)):
        bad = capi.mgh_default_params()
        bad.restart, bad.deflate = restart, k
        with pytest.raises(capi.MGHError) as e:
            capi.mgh_workspace_bytes(bad)
        assert e.value.status == status
    mixed = capi.mgh_default_params()
    mixed.precision, mixed.arnoldi, mixed.deflate = capi.MGH_PREC_MIXED32, capi.MGH_ARNOLDI_FP64, 10
    assert capi.mgh_workspace_bytes(mixed) > 0
    for arnoldi, krylov in ((capi.MGH_ARNOLDI_DF, capi.MGH_KRYLOV_FGMRES), (capi.MGH_ARNOLDI_FP64, capi.MGH_KRYLOV_BICGSTAB)):
        bad = capi.mgh_default_params()
        bad.precision, bad.arnoldi, bad.krylov, bad.deflate = capi.MGH_PREC_MIXED32, arnoldi, krylov, 4
        bad.restart = 8
        with pytest.raises(capi.MGHError) as e:
            capi.mgh_workspace_bytes(bad)
        assert e.value.status == capi.MGH_NOT_SUPPORTED
