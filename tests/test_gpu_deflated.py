"""Flexible GMRES with deflated restarting on the CUDA path (the deflate parameter: k harmonic Ritz
vectors kept across restarts; GMRES-DR of Morgan 2002 in the flexible form of Giraud et al. 2010).

Checks against the oracle: the converged field against the exact sparse solve, the step count
against the oracle's fgmres_dr with the same multigrid preconditioner (same method; the device's
conditional second Gram-Schmidt pass and its residual taken from the true residual change the
rounding, not the iteration), on the FP64 path and on the mixed path (FP32 cycle, native FP64
Arnoldi); that deflation needs fewer steps than plain restarts on the strong-scattering recipe;
and that a batch with a zero right-hand side and several angles gives each right-hand side its own
solution.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda
from oracle.krylov import fgmres_dr

pytestmark = pytest.mark.gpu


def _w(**kw):
    # 52 x 45 extended grid: two reduction blocks per right-hand side with a ragged last block
    return W.Workload("dr", 40, 33, 6, 8.0, 2, -30.0, 30.0, "ellipses", 11, levels=3, nu1=1, nu2=1,
                      restart=8, tol=1e-10, **kw)


@pytest.mark.parametrize("precision,arnoldi,bound", [("fp64", "auto", 1e-8), ("mixed32", "fp64", 1e-5)])
def test_deflated_fgmres_matches_the_oracle(precision, arnoldi, bound):
    torch = torch_cuda()
    w = _w(precision=precision)
    m, k = 8, 4
    p, f, o = oracle_solver(w, tol=1e-10)
    th = W.angles(w)[:2]
    b = np.stack([O.rhs(p, f, t) for t in th])
    s = make_solver(w, B=2, maxit=3000, arnoldi=arnoldi, deflate=k)
    s.set_contrast(torch.from_numpy(f).cuda())
    x, infos = s.solve(torch.from_numpy(b).cuda())
    x = x.cpu().numpy()
    for q in range(2):
        assert infos[q]["converged"] and infos[q]["rel_residual"] <= 1e-10, infos
        assert rel(x[q], O.direct_solve(p, o.D, b[q])) < bound
        _, ref = fgmres_dr(o.apply_A, o.M, b[q], 1e-10, m, k, 3000)
        slack = max(2 * m, int(0.1 * ref.iterations))
        assert abs(infos[q]["iterations"] - ref.iterations) <= slack, (infos[q], ref.iterations)
    s.close()


def test_batch_with_a_zero_right_hand_side_and_solo_runs():
    torch = torch_cuda()
    w = _w(precision="fp64")
    p, f, o = oracle_solver(w, tol=1e-10)
    b0 = O.rhs(p, f, 0.35)
    b = np.stack([b0, np.zeros_like(b0), O.rhs(p, f, -0.8)])
    s = make_solver(w, B=3, maxit=3000, deflate=3)
    s.set_contrast(torch.from_numpy(f).cuda())
    x, infos = s.solve(torch.from_numpy(b).cuda())
    x = x.cpu().numpy()
    assert infos[1]["converged"] and infos[1]["iterations"] == 0 and np.all(x[1] == 0)
    solo = make_solver(w, B=1, maxit=3000, deflate=3)
    solo.set_contrast(torch.from_numpy(f).cuda())
    for q in (0, 2):
        assert infos[q]["converged"], infos
        xs, info_s = solo.solve(torch.from_numpy(b[q:q + 1]).cuda())
        assert abs(info_s[0]["iterations"] - infos[q]["iterations"]) <= 2, (info_s, infos[q])
        ref = O.direct_solve(p, o.D, b[q])
        assert rel(x[q], ref) < 1e-8 and rel(xs.cpu().numpy()[0], ref) < 1e-8
    s.close()
    solo.close()


@pytest.mark.parametrize("precision,arnoldi", [("fp64", "auto"), ("mixed32", "fp64")])
def test_deflation_beats_plain_restarts_on_the_strong_scattering_recipe(precision, arnoldi):
    """The cell recipe at 128^2 + 8 (n/n_b to 1.5, 12 points per wavelength, kappa = 1 + 1j):
    FGMRES-DR(8, 4) needs fewer steps than FGMRES(8) and meets the exact solve."""
    torch = torch_cuda()
    w = replace(W.WORKLOADS["cell1120"], name="cell128", nx_int=128, ny_int=128, abl=8, levels=4,
                shift_im=1.0, krylov="fgmres", restart=8, tol=1e-8, precision=precision, nu1=2, nu2=2)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    b = O.rhs(p, f, 0.3)[None]
    steps = {}
    for k in (0, 4):
        s = make_solver(w, B=1, maxit=6000, arnoldi=arnoldi, deflate=k)
        s.set_contrast(torch.from_numpy(f).cuda())
        x, infos = s.solve(torch.from_numpy(b).cuda())
        assert infos[0]["converged"], (k, infos)
        steps[k] = infos[0]["iterations"]
        if k:
            o = O.MGHSolver(p, f, w.levels, 2, 2, 0.8, complex(w.shift_re, w.shift_im), 8, 1e-8)
            ref = O.direct_solve(p, o.D, b[0])
            assert rel(x.cpu().numpy()[0], ref) < (1e-6 if precision == "fp64" else 1e-5)
        s.close()
    assert steps[4] < 0.8 * steps[0], steps


@pytest.mark.parametrize("precision,arnoldi", [("fp64", "auto"), ("mixed32", "fp64")])
def test_fallback_restart_equals_plain_restarts(precision, arnoldi, monkeypatch):
    """When the host routine gives up, a right-hand side restarts plainly from its true residual
    (copied from W into basis slot 0).  With every deflated restart sent down that path
    (MGH_DEFLATE_FORCE_PLAIN=1) the solve is the plain-restart engine's, bit for bit."""
    torch = torch_cuda()
    w = _w(precision=precision)
    p, f, o = oracle_solver(w, tol=1e-10)
    b = np.stack([O.rhs(p, f, t) for t in W.angles(w)[:2]])
    res = {}
    for k, force in ((0, "0"), (4, "1")):
        monkeypatch.setenv("MGH_DEFLATE_FORCE_PLAIN", force)
        s = make_solver(w, B=2, maxit=3000, arnoldi=arnoldi, deflate=k)
        s.set_contrast(torch.from_numpy(f).cuda())
        x, infos = s.solve(torch.from_numpy(b).cuda())
        res[k] = (x.cpu().numpy(), [i["iterations"] for i in infos], [i["converged"] for i in infos])
        s.close()
    assert all(res[4][2]) and res[4][1] == res[0][1], (res[4][1], res[0][1])
    np.testing.assert_array_equal(res[4][0], res[0][0])
