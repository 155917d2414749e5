"""Host side of the IDR(s) engine (krylov MGH_KRYLOV_IDRS), no GPU needed: parameter checks of the
C ABI through mgh_workspace_bytes, and the shadow space both sides draw (workloads.idr_shadow,
random signs from MurmurHash3's 32-bit finaliser), pinned to the finaliser's published value and
to the properties the method needs of it."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.krylov import idrs


@pytest.fixture(scope="module")
def capi():
    import os
    from paper_2107_03679_gb300 import build
    if not os.path.exists(build.LIB):
        import __graft_entry__ as g
        g.build()
    from paper_2107_03679_gb300 import capi as c
    return c


def test_fmix32_published_values():
    assert int(W.fmix32(np.array([0], np.uint32))[0]) == 0
    assert int(W.fmix32(np.array([1], np.uint32))[0]) == 0x514E28B7


def test_shadow_space_entries_and_nesting():
    P8 = W.idr_shadow(4096, 8)
    assert set(np.unique(P8.real)) == {-1.0, 1.0} and set(np.unique(P8.imag)) == {-1.0, 1.0}
    np.testing.assert_array_equal(W.idr_shadow(4096, 3), P8[:, :3])
    G = P8.conj().T @ P8 / (2 * 4096)
    assert np.allclose(np.diag(G), 1.0)
    assert np.max(np.abs(G - np.eye(8))) < 0.1          # generic: close to orthogonal columns
    assert abs(P8.real.mean()) < 0.05 and abs(P8.imag.mean()) < 0.05
    with pytest.raises(ValueError):
        W.idr_shadow(10, 0)


def test_oracle_idrs_with_the_shared_shadow_space_reaches_the_direct_solve():
    w = W.small_workload(n_int=24, abl=4, seed=5, levels=3)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    s = O.MGHSolver(p, f, levels=3, nu1=1, nu2=1, tol=1e-30)
    b = O.rhs(p, f, 0.4)
    x, info = idrs(s.apply_A, s.M, b, 1e-12, 4, 600, shadow=W.idr_shadow(p.nx * p.ny, 4))
    assert info.converged
    ref = O.direct_solve(p, s.D, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_idrs_parameter_validation(capi):
    p = capi.mgh_default_params()
    assert p.idr_s == 4
    p.krylov, p.restart = capi.MGH_KRYLOV_IDRS, 10
    assert capi.mgh_workspace_bytes(p) > 0
    for s, restart in ((4, 9), (0, 10), (9, 20), (-1, 10)):
        bad = capi.mgh_default_params()
        bad.krylov, bad.idr_s, bad.restart = capi.MGH_KRYLOV_IDRS, s, restart
        with pytest.raises(capi.MGHError) as e:
            capi.mgh_workspace_bytes(bad)
        assert e.value.status == capi.MGH_INVALID_ARG
    ok = capi.mgh_default_params()
    ok.krylov, ok.idr_s, ok.restart, ok.precision = capi.MGH_KRYLOV_IDRS, 8, 18, capi.MGH_PREC_MIXED32
    assert capi.mgh_workspace_bytes(ok) > 0
    for field, value in (("precision", capi.MGH_PREC_MIXED16), ("deflate", 4)):
        bad = capi.mgh_default_params()
        bad.krylov, bad.restart = capi.MGH_KRYLOV_IDRS, 10
        setattr(bad, field, value)
        if field == "precision":
            bad.arnoldi = capi.MGH_ARNOLDI_SSTEP
        with pytest.raises(capi.MGHError) as e:
            capi.mgh_workspace_bytes(bad)
        assert e.value.status == capi.MGH_NOT_SUPPORTED
    fg = capi.mgh_default_params()
    fg.idr_s = 0                                          # read only with krylov MGH_KRYLOV_IDRS
    assert capi.mgh_workspace_bytes(fg) > 0
