"""FP16 storage on the fine level (MGH_PREC_MIXED16): the level-0 iterate between pre- and
post-smoothing and the preconditioned vectors Z stored as complex FP16, FP32 arithmetic, s-step
FGMRES(8).  Flexible GMRES forms the iterate from the stored z_k and their products A z_k, so the
rounding changes only the preconditioner (the oracle pin
test_flexible_gmres_tolerates_fp16_rounded_preconditioned_vectors): refined to a tight residual the
fields meet the FP64 references within the mixed-precision tolerance 1e-5, and the step counts stay
those of the FP32-stored path."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def to_t(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ragged16(tol=1e-10, **kw):
    # 88 x 71 extended grid: even width (FP16 pairs), odd height, several strips and a ragged one
    return W.Workload("ragged16", 70, 53, 9, 8.0, 3, -50.0, 40.0, "ellipses", 11, levels=4, nu1=2, nu2=2,
                      restart=8, precision="mixed16", tol=tol, **kw)


def test_mixed16_solve_matches_direct_solve_and_fp32_storage_steps():
    torch = torch_cuda()
    w = ragged16()
    p, f, o = oracle_solver(w)
    th = W.angles(w)
    b = np.stack([O.rhs(p, f, t) for t in th])
    out = {}
    for prec in ("mixed16", "mixed32"):
        s = make_solver(w, B=3, maxit=6000, precision=prec)
        assert s.arnoldi == "sstep"
        s.set_contrast(to_t(f, torch))
        x, infos = s.solve(to_t(b, torch))
        assert all(i["converged"] and i["rel_residual"] <= 1e-10 for i in infos), (prec, infos)
        out[prec] = (x.cpu().numpy(), [i["iterations"] for i in infos])
        s.close()
    for q in range(3):
        ref = O.direct_solve(p, o.D, b[q])
        assert rel(out["mixed16"][0][q], ref) < 1e-5
        true = np.linalg.norm(b[q] - o.apply_A(out["mixed16"][0][q])) / np.linalg.norm(b[q])
        assert true <= 1e-10 * (1 + 1e-6)
    for a, c in zip(out["mixed16"][1], out["mixed32"][1]):
        assert abs(a - c) <= max(8, 0.05 * c), (out["mixed16"][1], out["mixed32"][1])


def test_mixed16_gradient_matches_oracle():
    torch = torch_cuda()
    w = W.Workload("grad16", 70, 53, 9, 8.0, 4, -50.0, 40.0, "gt_ellipse", 4, levels=4, nu1=2, nu2=2,
                   restart=8, precision="mixed16", tol=1e-10)
    p, f_gt, o = oracle_solver(w, tol=1e-13)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    y = O.sample(o.forward(th)[0], rec) + W.complex_noise((len(th), rec.size), 0.01, 4)
    f = 0.6 * f_gt
    _, _, o2 = oracle_solver(w, tol=1e-13, f=f)
    loss_ref, g_ref, _ = o2.gradient(th, rec, y)
    s = make_solver(w, B=len(th), maxit=6000)
    s.set_contrast(to_t(f, torch))
    d_th = to_t(th, torch)
    u, inf_f = s.forward(d_th)
    _, G, loss = s.misfit(u, to_t(y, torch), to_t(rec, torch))
    g, inf_a = s.gradient(d_th, u, G)
    assert all(i["converged"] for i in inf_f + inf_a)
    assert loss == pytest.approx(loss_ref, rel=1e-8)
    assert rel(g.cpu().numpy(), g_ref) < 1e-5


def test_mixed16_full_size_field_matches_fp64_path():
    """The batched workload (512^2 + 32 layer, 6 levels): two angles with FP16 storage and with the
    plain FP64 path, both to relative residual 1e-8; fields within 1e-5, steps within 5 % of the
    FP32-stored path's."""
    torch = torch_cuda()
    w = W.WORKLOADS["ellipses576"]
    f = W.phantom(w)
    th = W.angles(w)[[0, 59]]
    out = {}
    for prec in ("mixed16", "mixed32", "fp64"):
        s = make_solver(w, B=2, maxit=6000, precision=prec, tol=1e-8)
        s.set_contrast(to_t(f, torch))
        u, infos = s.forward(to_t(th, torch))
        assert all(i["converged"] for i in infos), (prec, infos)
        out[prec] = (u.cpu().numpy(), [i["iterations"] for i in infos])
        s.close()
    d = max(rel(out["mixed16"][0][q], out["fp64"][0][q]) for q in range(2))
    assert d < 1e-5, d
    for a, c in zip(out["mixed16"][1], out["mixed32"][1]):
        assert abs(a - c) <= 0.05 * c, (out["mixed16"][1], out["mixed32"][1])


def test_mixed16_configurations_it_does_not_cover_are_refused():
    torch_cuda()
    from paper_2107_03679_gb300 import capi
    cases = [dict(w=W.Workload("odd16", 41, 30, 6, 8.0, 1, 0, 0, "ellipses", 3, levels=3, nu1=1, nu2=1,
                               restart=8, precision="mixed16"), kw={}),          # odd width 53
             dict(w=ragged16(), kw=dict(krylov="bicgstab")),
             dict(w=ragged16(), kw=dict(arnoldi="df"))]
    for c in cases:
        with pytest.raises(capi.MGHError) as e:
            make_solver(c["w"], B=1, **c["kw"])
        assert e.value.status == capi.MGH_NOT_SUPPORTED
