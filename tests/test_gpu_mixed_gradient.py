"""Parity of the gradient path that the batched bench times: mixed precision (FP32 multigrid
cycle, s-step FGMRES(8) cycles with an FP32 basis, double-float iterate, FP64-verified acceptance)
for the forward and the adjoint solves, then the gradient of Prop. 1 (Sec. V).

Tolerances follow the reading that two solutions converged to relative residual tau differ by at
most cond(A) tau: the mixed path is refined to a tight residual and must then meet the FP64 oracle
within the mixed-precision tolerance 1e-5 (relative L2), the bound stated for mixed results.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def to_t(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ragged_gradient_workload(tol):
    # 70 x 53 interior + 9-cell layer (88 x 71): several wavefront strips and a ragged last one
    return W.Workload("gradmix", 70, 53, 9, 8.0, 4, -50.0, 40.0, "gt_ellipse", 4, levels=4, nu1=2, nu2=2,
                      restart=8, precision="mixed32", tol=tol)


def _data(w, o, th, rec):
    """Receiver data of the ground-truth contrast (oracle forward, FP64) plus 1 % noise."""
    return O.sample(o.forward(th)[0], rec) + W.complex_noise((len(th), rec.size), 0.01, 4)


def test_mixed_sstep_gradient_matches_oracle_on_ragged_grid():
    """mgh_gradient with precision mixed32 and the s-step engine (the bench's configuration) on a
    ragged grid: forward and adjoint solves refined to a relative residual of 1e-10, the gradient
    within 1e-5 of the oracle's (forward and adjoint solves at 1e-13) and the loss within 1e-8."""
    torch = torch_cuda()
    w = _ragged_gradient_workload(1e-10)
    p, f_gt, o = oracle_solver(w, tol=1e-13)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    y = _data(w, o, th, rec)
    f = 0.6 * f_gt
    _, _, o2 = oracle_solver(w, tol=1e-13, f=f)
    loss_ref, g_ref, _ = o2.gradient(th, rec, y)
    s = make_solver(w, B=len(th), maxit=6000, arnoldi="sstep")
    assert s.arnoldi == "sstep" and s.precision == "mixed32"
    s.set_contrast(to_t(f, torch))
    d_th = to_t(th, torch)
    u, inf_f = s.forward(d_th)
    _, G, loss = s.misfit(u, to_t(y, torch), to_t(rec, torch))
    g, inf_a = s.gradient(d_th, u, G)
    assert all(i["converged"] and i["rel_residual"] <= 1e-10 for i in inf_f + inf_a), inf_f + inf_a
    assert loss == pytest.approx(loss_ref, rel=1e-8)
    assert rel(g.cpu().numpy(), g_ref) < 1e-5, rel(g.cpu().numpy(), g_ref)


def _sigma_min(A):
    """Smallest singular value of a sparse matrix by inverse iteration on A^H A (sparse LU)."""
    lu = spla.splu(A.tocsc())
    x = np.random.default_rng(0).standard_normal(A.shape[0]) + 0j
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(60):
        y = lu.solve(lu.solve(x, trans="H"))      # A^-1 A^-H x = (A^H A)^-1 x
        lam_new = np.linalg.norm(y)
        x = y / lam_new
        if abs(lam_new - lam) <= 1e-10 * lam_new:
            break
        lam = lam_new
    return 1.0 / np.sqrt(lam_new)


def test_mixed_sstep_gradient_twenty_directions_against_central_differences():
    """Twenty seeded directions d: the mixed-precision gradient's g.d against central differences
    of the loss, both computed on the GPU's mixed path with every solve stopped at relative
    residual tau = 1e-10.

    Tolerance from the stopping residual: a field solved to ||b - A u|| <= tau ||b|| is within
    ||A^-1|| tau ||b|| of the exact one, so each loss evaluation is off by at most
    dL = sum_q ||S u_q - y_q|| ||A^-1|| tau ||b_q|| (+ a second-order term), and the difference
    quotient by at most dL / eps.  The test takes ||A^-1|| = 1/sigma_min(A) of this grid (inverse
    iteration, doubled for safety), adds
    the central-difference truncation (relative 1e-6 at eps = 1e-4) and the gradient's own bound
    (1e-5 relative, from the oracle comparison above)."""
    torch = torch_cuda()
    tau, eps = 1e-10, 1e-4
    w = _ragged_gradient_workload(tau)
    p, f_gt, o = oracle_solver(w, tol=1e-13)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    y = _data(w, o, th, rec)
    f = 0.6 * f_gt
    s = make_solver(w, B=len(th), maxit=6000, arnoldi="sstep")
    d_th, d_rec, d_y = to_t(th, torch), to_t(rec, torch), to_t(y, torch)

    def loss_at(ff):
        s.set_contrast(to_t(ff, torch))
        u, infos = s.forward(d_th)
        assert all(i["converged"] for i in infos)
        r, G, loss = s.misfit(u, d_y, d_rec)
        return u, r, G, loss

    u, r, G, loss = loss_at(f)
    g, _ = s.gradient(d_th, u, G)
    g = g.cpu().numpy()
    # loss error bound of one evaluation, from the stopping residual
    c = O.fine_coefficient(p, f)
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    inv_norm = 2.0 / _sigma_min(O.assemble_operator(D, p.h))   # x2: inverse iteration converges from above
    rn = np.linalg.norm(r.cpu().numpy(), axis=1)
    bn = np.array([np.linalg.norm(O.rhs(p, f, t)) for t in th])
    dL = float(np.sum(rn * inv_norm * tau * bn) + 0.5 * np.sum((inv_norm * tau * bn) ** 2))
    rng = np.random.default_rng(20)
    for _ in range(20):
        d = rng.standard_normal(f.shape)
        fd = (loss_at(f + eps * d)[3] - loss_at(f - eps * d)[3]) / (2 * eps)
        gd = float(np.sum(g * d))
        bound = 2 * dL / (2 * eps) + 1e-6 * abs(fd) + 1e-5 * np.linalg.norm(g) * np.linalg.norm(d)
        assert abs(gd - fd) <= bound, (gd, fd, bound)


def test_mixed_gradient_full_size_matches_fp64_path():
    """The bench configuration at full size (512^2 + 32 layer, 6 levels, FP32 cycle, s-step
    FGMRES(8)): two angles' forward + adjoint gradient on the mixed path and on the plain FP64
    path, every solve to relative residual 1e-8; the gradients agree within 1e-5 and the losses
    within 1e-8."""
    torch = torch_cuda()
    w = W.WORKLOADS["ellipses576"]
    f_gt = W.phantom(w)
    f = 0.9 * f_gt
    th = W.angles(w)[[0, 59]]
    rec = W.receivers(w, f_gt)
    d_th, d_rec = to_t(th, torch), to_t(rec, torch)
    out = {}
    y = None
    for prec in ("fp64", "mixed32"):
        s = make_solver(w, B=2, maxit=6000, precision=prec, tol=1e-8)
        if y is None:   # data: the ground truth's receiver samples (FP64 path)
            s.set_contrast(to_t(f_gt, torch))
            u_gt, _ = s.forward(d_th)
            y = s.sample(u_gt, d_rec)
        s.set_contrast(to_t(f, torch))
        u, inf_f = s.forward(d_th)
        _, G, loss = s.misfit(u, y, d_rec)
        g, inf_a = s.gradient(d_th, u, G)
        assert all(i["converged"] for i in inf_f + inf_a), (prec, inf_f + inf_a)
        out[prec] = (g.cpu().numpy(), loss, s.arnoldi)
        s.close()
    assert out["mixed32"][2] == "sstep"
    assert out["mixed32"][1] == pytest.approx(out["fp64"][1], rel=1e-8)
    assert rel(out["mixed32"][0], out["fp64"][0]) < 1e-5, rel(out["mixed32"][0], out["fp64"][0])
