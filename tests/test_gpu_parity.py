"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Sizes span several tiles of the V-cycle kernels with ragged tails in x and y (88 x 71 points:
tiles are 64 or 32 wide and 16 high) and ragged batches.  Tolerances:
  * FP64 pointwise kernels and FP64 multigrid cycles: relative L2 <= 1e-12 (rounding order only);
  * FP32 multigrid cycle: relative L2 <= 1e-5 against the FP64 cycle;
  * solves: both sides solved to a tight residual, fields within 1e-10 (FP64 path) and 1e-5
    (mixed path), per the reading that two converged solutions differ by at most cond(A)*tol.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def ragged(precision="fp64", levels=4, nu1=1, nu2=1, n_angles=3, **kw):
    w = W.Workload("ragged", 70, 53, 9, 8.0, n_angles, -50.0, 40.0, "ellipses", 11, levels=levels,
                   nu1=nu1, nu2=nu2, precision=precision, **kw)
    return w


def to_t(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_incident_field_and_rhs():
    torch = torch_cuda()
    w = ragged()
    s = make_solver(w, B=4)
    p, f, _ = oracle_solver(w)
    th = W.angles(w)
    s.set_contrast(to_t(f, torch))
    uin = s.incident_field(to_t(th, torch)).cpu().numpy()
    b = s.rhs(to_t(th, torch)).cpu().numpy()
    for q, t in enumerate(th):
        assert rel(uin[q], O.incident_field(p, t)) < 1e-12
        assert rel(b[q], O.rhs(p, f, t)) < 1e-12


def test_operator_apply():
    torch = torch_cuda()
    w = ragged()
    s = make_solver(w, B=4)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    x = W.random_field((3, p.ny, p.nx), 5)
    y = s.apply(to_t(x, torch)).cpu().numpy()
    for q in range(3):
        assert rel(y[q], o.apply_A(x[q])) < 1e-13


def test_hierarchy_coefficients():
    torch = torch_cuda()
    w = ragged(levels=4)
    s = make_solver(w, B=1)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    for l, lv in enumerate(o.M.hier):
        nx, ny, h = s.level_shape(l)
        assert (nx, ny) == (lv.nx, lv.ny) and h == lv.h
        c = s.level_coefficient(l).cpu().numpy()
        np.testing.assert_allclose(c, lv.c, rtol=1e-14, atol=0)


def test_coarse_solve():
    torch = torch_cuda()
    w = ragged(levels=4)
    s = make_solver(w, B=2)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    cl = o.M.hier[-1]
    b = W.random_field((2, cl.ny, cl.nx), 9)
    x = s.coarse_solve(to_t(b, torch)).cpu().numpy()
    for q in range(2):
        assert rel(x[q], o.M.coarse(b[q])) < 1e-12


@pytest.mark.parametrize("levels,nu1,nu2", [(2, 0, 0), (3, 1, 1), (4, 2, 2), (3, 2, 1), (4, 0, 3), (4, 4, 4)])
def test_vcycle_fp64(levels, nu1, nu2):
    torch = torch_cuda()
    w = ragged(levels=levels, nu1=nu1, nu2=nu2)
    if levels == 2:
        w = W.Workload("ragged2", 30, 21, 5, 8.0, 3, 0, 0, "ellipses", 12, levels=2, nu1=0, nu2=0,
                       precision="fp64")
    s = make_solver(w, B=4)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    b = W.random_field((3, p.ny, p.nx), 13)
    z = s.precondition(to_t(b, torch)).cpu().numpy()
    for q in range(3):
        assert rel(z[q], o.M(b[q])) < 1e-12, (q, rel(z[q], o.M(b[q])))


@pytest.mark.parametrize("nu", [1, 2])
def test_vcycle_mixed32(nu):
    torch = torch_cuda()
    w = ragged(levels=4, nu1=nu, nu2=nu, precision="mixed32")
    s = make_solver(w, B=3)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    b = W.random_field((3, p.ny, p.nx), 14)
    z = s.precondition(to_t(b, torch)).cpu().numpy()
    for q in range(3):
        assert rel(z[q], o.M(b[q])) < 1e-5


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-10), ("mixed32", 1e-10, 1e-5)])
def test_solve_matches_direct_solve(precision, tol, bound):
    torch = torch_cuda()
    w = ragged(precision=precision, levels=4, nu1=1, nu2=1, tol=tol)
    s = make_solver(w, B=4, maxit=3000)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    th = W.angles(w)
    b = np.stack([O.rhs(p, f, t) for t in th])
    x, infos = s.solve(to_t(b, torch))
    x = x.cpu().numpy()
    for q in range(len(th)):
        assert infos[q]["converged"] and infos[q]["rel_residual"] <= tol
        ref = O.direct_solve(p, o.D, b[q])
        assert rel(x[q], ref) < bound
        # the reported residual is the true FP64 residual of the returned field
        true = np.linalg.norm(b[q] - o.apply_A(x[q])) / np.linalg.norm(b[q])
        assert true <= tol * (1 + 1e-6)


@pytest.mark.parametrize("restart", [4, 10, 20])
def test_mixed_arnoldi_variants_agree(restart):
    """Double-float Arnoldi (FP32 pipes) and native-FP64 Arnoldi reach the same solution."""
    torch = torch_cuda()
    w = ragged(precision="mixed32", levels=4, nu1=1, nu2=1, tol=1e-10, restart=restart)
    p, f, o = oracle_solver(w)
    th = W.angles(w)
    b = np.stack([O.rhs(p, f, t) for t in th])
    out = {}
    for ar in ("df", "fp64"):
        s = make_solver(w, B=3, maxit=3000, arnoldi=ar)
        s.set_contrast(to_t(f, torch))
        x, infos = s.solve(to_t(b, torch))
        assert all(i["converged"] for i in infos), (ar, infos)
        out[ar] = (x.cpu().numpy(), [i["iterations"] for i in infos])
    for q in range(3):
        ref = O.direct_solve(p, o.D, b[q])
        assert rel(out["df"][0][q], ref) < 1e-5
        assert rel(out["df"][0][q], out["fp64"][0][q]) < 1e-5
    # same Krylov method: iteration counts within a few steps
    for a, c in zip(out["df"][1], out["fp64"][1]):
        assert abs(a - c) <= max(3, 0.1 * c)


@pytest.mark.parametrize("restart", [1, 4, 8])
def test_sstep_cycles_match_direct_solve_and_arnoldi(restart):
    """s-step cycles (monomial basis orthogonalised by the Cholesky factor of its Gram matrix)
    reach the direct solution, with the iteration counts of Arnoldi-based FGMRES(m): in exact
    arithmetic both minimise the residual over the same space in every cycle."""
    torch = torch_cuda()
    w = ragged(precision="mixed32", levels=4, nu1=1, nu2=1, tol=1e-10, restart=restart)
    p, f, o = oracle_solver(w)
    th = W.angles(w)
    b = np.stack([O.rhs(p, f, t) for t in th])
    out = {}
    for ar in ("df", "sstep"):
        s = make_solver(w, B=3, maxit=6000, arnoldi=ar)
        s.set_contrast(to_t(f, torch))
        x, infos = s.solve(to_t(b, torch))
        assert all(i["converged"] for i in infos), (ar, infos)
        out[ar] = (x.cpu().numpy(), [i["iterations"] for i in infos], [i["rel_residual"] for i in infos])
    for q in range(3):
        ref = O.direct_solve(p, o.D, b[q])
        xs = out["sstep"][0][q]
        assert rel(xs, ref) < 1e-5
        true = np.linalg.norm(b[q] - o.apply_A(xs)) / np.linalg.norm(b[q])
        assert true <= 1e-10 * (1 + 1e-6) and abs(true - out["sstep"][2][q]) <= 1e-3 * 1e-10
    for a, c in zip(out["sstep"][1], out["df"][1]):
        assert abs(a - c) <= max(3, 0.1 * c)


def test_sstep_zero_rhs_maxit_and_oracle_iterations():
    """b = 0 gives x = 0 in zero steps; maxit caps the steps even inside a cycle; and the step
    count to 1e-8 matches the oracle's FGMRES(8) on the same problem."""
    torch = torch_cuda()
    w = ragged(precision="mixed32", levels=4, nu1=1, nu2=1, restart=8, tol=1e-8)
    p, f, o = oracle_solver(w, tol=1e-8, restart=8)
    s = make_solver(w, B=3, maxit=2, arnoldi="sstep")
    s.set_contrast(to_t(f, torch))
    b = np.zeros((3, p.ny, p.nx), dtype=np.complex128)
    b[1] = O.rhs(p, f, 0.3)
    x, infos = s.solve(to_t(b, torch), x0=to_t(W.random_field((3, p.ny, p.nx), 1), torch))
    x = x.cpu().numpy()
    assert np.all(x[0] == 0) and np.all(x[2] == 0)
    assert infos[0]["iterations"] == 0 and infos[0]["converged"]
    assert not infos[1]["converged"] and infos[1]["iterations"] == 2
    s = make_solver(w, B=1, maxit=6000, arnoldi="sstep")
    s.set_contrast(to_t(f, torch))
    x, infos = s.solve(to_t(b[1:2], torch))
    _, ref = o.solve(b[1])
    assert infos[0]["converged"] and ref.converged
    assert abs(infos[0]["iterations"] - ref.iterations) <= max(5, 0.1 * ref.iterations), (infos, ref.iterations)


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-10), ("mixed32", 1e-10, 1e-5)])
def test_bicgstab_matches_direct_solve_and_oracle(precision, tol, bound):
    """Bi-CGSTAB of Alg. 3 (two multigrid cycles per iteration): the direct solution within the
    path's tolerance, the true residual it reports, and the oracle's step count (FP64 path: same
    arithmetic up to rounding order; mixed path: FP32 cycle)."""
    torch = torch_cuda()
    w = ragged(precision=precision, levels=4, nu1=1, nu2=1, tol=tol, restart=8)
    s = make_solver(w, B=3, maxit=3000, krylov="bicgstab")
    p, f, o = oracle_solver(w, tol=tol, krylov="bicgstab")
    s.set_contrast(to_t(f, torch))
    th = W.angles(w)
    b = np.stack([O.rhs(p, f, t) for t in th])
    x, infos = s.solve(to_t(b, torch))
    x = x.cpu().numpy()
    for q in range(len(th)):
        assert infos[q]["converged"], infos
        ref = O.direct_solve(p, o.D, b[q])
        assert rel(x[q], ref) < bound
        true = np.linalg.norm(b[q] - o.apply_A(x[q])) / np.linalg.norm(b[q])
        assert true <= tol * (1 + 1e-6)
        _, info_ref = o.solve(b[q])
        slack = max(4, 0.05 * info_ref.iterations) if precision == "fp64" else max(8, 0.15 * info_ref.iterations)
        assert abs(infos[q]["iterations"] - info_ref.iterations) <= slack, (infos[q], info_ref.iterations)


def test_bicgstab_zero_rhs_and_maxit():
    torch = torch_cuda()
    w = ragged(precision="mixed32", levels=4, nu1=1, nu2=1, restart=8)
    p, f, o = oracle_solver(w)
    s = make_solver(w, B=3, maxit=2, krylov="bicgstab")
    s.set_contrast(to_t(f, torch))
    b = np.zeros((3, p.ny, p.nx), dtype=np.complex128)
    b[1] = O.rhs(p, f, 0.3)
    x, infos = s.solve(to_t(b, torch), x0=to_t(W.random_field((3, p.ny, p.nx), 1), torch))
    x = x.cpu().numpy()
    assert np.all(x[0] == 0) and np.all(x[2] == 0)
    assert infos[0]["iterations"] == 0 and infos[0]["converged"]
    assert not infos[1]["converged"] and infos[1]["iterations"] == 2


def test_forward_matches_oracle_forward():
    torch = torch_cuda()
    w = ragged(precision="fp64", tol=1e-11)
    s = make_solver(w, B=3, maxit=3000)
    p, f, o = oracle_solver(w, tol=1e-12)
    s.set_contrast(to_t(f, torch))
    th = W.angles(w)
    u, infos = s.forward(to_t(th, torch))
    u_ref, _ = o.forward(th)
    assert rel(u.cpu().numpy(), u_ref) < 1e-9
    crop = s.crop(u).cpu().numpy()
    np.testing.assert_array_equal(crop, O.crop(p, u.cpu().numpy()))


def test_disk160_workload_fp64():
    """The plain single-solve workload: 128^2 + 16 layer, disk r=20, one wave along +x, FP64,
    GMRES(20), shift 1+0.5i, 4 levels, 2+2 sweeps, tol 1e-8."""
    torch = torch_cuda()
    w = W.WORKLOADS["disk160"]
    s = make_solver(w, B=1, maxit=4000)
    p, f, o = oracle_solver(w, tol=w.tol)
    s.set_contrast(to_t(f, torch))
    th = W.angles(w)
    u, infos = s.forward(to_t(th, torch))
    u = u.cpu().numpy()[0]
    b = O.rhs(p, f, th[0])
    assert infos[0]["converged"]
    true = np.linalg.norm(b - o.apply_A(u)) / np.linalg.norm(b)
    assert true <= w.tol * (1 + 1e-6)
    _, info_ref = o.solve(b)
    # same method, same arithmetic up to rounding and Gram-Schmidt variant
    assert abs(infos[0]["iterations"] - info_ref.iterations) <= max(5, 0.05 * info_ref.iterations)
    ref = O.direct_solve(p, o.D, b)
    assert rel(u, ref) < 1e-5


def test_zero_rhs_and_maxit():
    torch = torch_cuda()
    from paper_2107_03679_gb300 import capi
    w = ragged()
    s = make_solver(w, B=3, maxit=2)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    b = np.zeros((3, p.ny, p.nx), dtype=np.complex128)
    b[1] = O.rhs(p, f, 0.3)
    x, infos = s.solve(to_t(b, torch), x0=to_t(W.random_field((3, p.ny, p.nx), 1), torch))
    x = x.cpu().numpy()
    assert np.all(x[0] == 0) and np.all(x[2] == 0)
    assert infos[0]["iterations"] == 0 and infos[0]["converged"]
    assert not infos[1]["converged"] and infos[1]["iterations"] == 2
    with pytest.raises(capi.MGHError):
        capi.mgh_solve(s._h, capi._ptr(to_t(b, torch)), 3, capi._ptr(to_t(b.copy(), torch)),
                       allow_not_converged=False)


def test_sample_scatter_misfit():
    torch = torch_cuda()
    w = ragged()
    s = make_solver(w, B=3)
    p, f, _ = oracle_solver(w)
    u = W.random_field((3, p.ny, p.nx), 2)
    rec = W.receivers(w, f)
    y = W.random_field((3, rec.size), 3)
    ut, rt, yt = to_t(u, torch), to_t(rec, torch), to_t(y, torch)
    np.testing.assert_array_equal(s.sample(ut, rt).cpu().numpy(), O.sample(u, rec))
    r, G, loss = s.misfit(ut, yt, rt)
    r_ref, loss_ref = O.misfit(O.sample(u, rec), y)
    np.testing.assert_array_equal(r.cpu().numpy(), r_ref)
    assert loss == pytest.approx(loss_ref, rel=1e-13)
    G_ref = np.zeros((3, p.ny * p.nx), dtype=np.complex128)
    G_ref[:, rec] = r_ref
    np.testing.assert_array_equal(G.cpu().numpy().reshape(3, -1), G_ref)
    np.testing.assert_array_equal(s.scatter(r, rt).cpu().numpy(), G.cpu().numpy())


def _grad_problem():
    w = W.Workload("gradsmall", 24, 20, 6, 8.0, 3, -40.0, 40.0, "gt_ellipse", 4, levels=3, nu1=1, nu2=1,
                   precision="fp64", tol=1e-12)
    return w


def test_gradient_matches_oracle():
    torch = torch_cuda()
    w = _grad_problem()
    s = make_solver(w, B=3, maxit=3000)
    p, f_gt, o = oracle_solver(w, tol=1e-13)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    y = O.sample(o.forward(th)[0], rec) + W.complex_noise((len(th), rec.size), 0.01, 4)
    f = 0.5 * f_gt
    _, _, o2 = oracle_solver(w, tol=1e-13, f=f)
    loss_ref, g_ref, _ = o2.gradient(th, rec, y)
    s.set_contrast(to_t(f, torch))
    u, _ = s.forward(to_t(th, torch))
    _, G, loss = s.misfit(u, to_t(y, torch), to_t(rec, torch))
    g, infos = s.gradient(to_t(th, torch), u, G)
    assert loss == pytest.approx(loss_ref, rel=1e-9)
    assert rel(g.cpu().numpy(), g_ref) < 1e-8


def test_autograd_function_matches_finite_differences():
    torch = torch_cuda()
    from paper_2107_03679_gb300 import scattered_field
    w = _grad_problem()
    s = make_solver(w, B=3, maxit=3000)
    _, f_gt, o = oracle_solver(w, tol=1e-13)
    th = to_t(W.angles(w), torch)
    rec = to_t(W.receivers(w, f_gt), torch)
    y = to_t(O.sample(o.forward(W.angles(w))[0], W.receivers(w, f_gt)), torch)
    f = to_t(0.5 * f_gt, torch).requires_grad_(True)

    def loss_of(ff):
        u = scattered_field(ff, s, th, rec)
        return 0.5 * (u - y).abs().pow(2).sum()

    L = loss_of(f)
    L.backward()
    g = f.grad.detach()
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = to_t(rng.standard_normal(tuple(f.shape)), torch)
        eps = 1e-5
        with torch.no_grad():
            fd = (loss_of(f + eps * d) - loss_of(f - eps * d)) / (2 * eps)
        assert float((g * d).sum()) == pytest.approx(float(fd), rel=1e-6)


@pytest.mark.parametrize("arnoldi", ["df", "sstep"])
def test_ellipses576_full_size_residual_property(arnoldi):
    """Full-size batched mixed-precision forward (512^2 + 32 layer, 60 angles, FP32 V-cycle with
    6 levels, FGMRES(8) with double-float Arnoldi or s-step cycles, tol 1e-6), the launch
    configuration the bench times.  The oracle recomputes the true FP64 residual of sampled
    returned fields."""
    torch = torch_cuda()
    w = W.WORKLOADS["ellipses576"]
    s = make_solver(w, B=w.n_angles, maxit=5000, arnoldi=arnoldi)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    s.set_contrast(to_t(f, torch))
    th = W.angles(w)
    u, infos = s.forward(to_t(th, torch))
    assert all(i["converged"] for i in infos)
    c = O.fine_coefficient(p, f)
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    for q in [0, 29, 59]:
        uq = u[q].cpu().numpy()
        b = O.rhs(p, f, th[q])
        true = np.linalg.norm(b - O.apply_operator(D, uq, p.h)) / np.linalg.norm(b)
        assert true <= w.tol * (1 + 1e-6), (q, true)
        assert abs(true - infos[q]["rel_residual"]) <= 1e-3 * w.tol


def test_ellipses576_mixed_field_matches_fp64_path():
    """The bench configuration's field error: two angles of the full-size workload solved by the
    mixed path (FP32 cycle, s-step cycles) and by the plain FP64 path, both to a true relative
    residual of 1e-8; the two fields agree to well within the mixed tolerance of 1e-5.  The
    measured difference is written to $MGH_TEST_REPORT_DIR/mixed_vs_fp64_ellipses576.txt when that
    variable names a directory."""
    torch = torch_cuda()
    w = W.WORKLOADS["ellipses576"]
    f = W.phantom(w)
    th = W.angles(w)[[0, 59]]
    out = {}
    for prec in ("mixed32", "fp64"):
        s = make_solver(w, B=2, maxit=5000, precision=prec, tol=1e-8)
        s.set_contrast(to_t(f, torch))
        u, infos = s.forward(to_t(th, torch))
        assert all(i["converged"] for i in infos), (prec, infos)
        out[prec] = u.cpu().numpy()
        s.close()
    d = max(rel(out["mixed32"][q], out["fp64"][q]) for q in range(2))
    assert d < 1e-5, d
    import os
    report = os.environ.get("MGH_TEST_REPORT_DIR")
    if report and os.path.isdir(report):
        with open(os.path.join(report, "mixed_vs_fp64_ellipses576.txt"), "w") as fh:
            fh.write(f"{d:.3e}\n")


def test_gradient_twenty_directions_against_central_differences():
    """Differentiation check of the data-term gradient on 20 seeded random directions: the CUDA
    forward/adjoint gradient (FP64, tight tolerance) against central differences of the loss
    computed with the CUDA forward solves, and against the oracle gradient."""
    torch = torch_cuda()
    w = W.Workload("fd20", 48, 48, 6, 8.0, 6, -60.0, 60.0, "gt_ellipse", 4, levels=3, nu1=2, nu2=2,
                   precision="fp64", tol=1e-12)
    s = make_solver(w, B=6, maxit=5000)
    p, f_gt, o = oracle_solver(w, tol=1e-13)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    y = O.sample(o.forward(th)[0], rec) + W.complex_noise((len(th), rec.size), 0.01, 4)
    f = 0.7 * f_gt
    d_th, d_rec, d_y = to_t(th, torch), to_t(rec, torch), to_t(y, torch)

    def loss_at(ff):
        s.set_contrast(to_t(ff, torch))
        u, infos = s.forward(d_th)
        assert all(i["converged"] for i in infos)
        return s.misfit(u, d_y, d_rec)

    _, G, loss = loss_at(f)
    u, _ = s.forward(d_th)
    g, _ = s.gradient(d_th, u, G)
    g = g.cpu().numpy()
    _, _, o2 = oracle_solver(w, tol=1e-13, f=f)
    _, g_ref, _ = o2.gradient(th, rec, y)
    assert rel(g, g_ref) < 1e-8
    rng = np.random.default_rng(20)
    eps = 1e-5
    for _ in range(20):
        d = rng.standard_normal(f.shape)
        fd = (loss_at(f + eps * d)[2] - loss_at(f - eps * d)[2]) / (2 * eps)
        assert float(np.sum(g * d)) == pytest.approx(fd, rel=1e-5, abs=1e-10)
