"""Several handles driven concurrently (one stream and one host thread each): the multi-frequency
data term and gradient against the FP64 oracle, and against the same handles run one at a time.

Two frequencies (5 and 8 GHz scaled to 8 points per wavelength at the higher one) on a 70 x 53
interior; FP64 path at residual 1e-12 against the oracle at 1e-13: losses within 1e-9, gradients
within 1e-8 (the bound of the single-frequency gradient test).  Running the handles concurrently
changes no arithmetic: the result equals the sequential one to 1e-13.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def to_t(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_multifrequency_gradient_matches_oracle_and_sequential_runs():
    torch = torch_cuda()
    from paper_2107_03679_gb300 import Solver
    from paper_2107_03679_gb300.multi import MultiFrequency
    base = W.Workload("mf", 70, 53, 9, 8.0, 2, -40.0, 30.0, "gt_ellipse", 4, levels=4, nu1=1, nu2=1,
                      precision="fp64", tol=1e-12)
    ws = W.multifrequency_workloads(base, freqs=(5.0, 8.0))
    f_gt = W.phantom(base)
    th = W.angles(base)
    rec = W.receivers(base, f_gt)
    f = 0.5 * f_gt
    ys, loss_ref, g_ref = [], 0.0, np.zeros_like(f)
    for i, w in enumerate(ws):
        _, _, o = oracle_solver(w, tol=1e-13, f=f_gt)
        y = O.sample(o.forward(th)[0], rec) + W.complex_noise((len(th), rec.size), 0.01, 20 + i)
        ys.append(y)
        _, _, o2 = oracle_solver(w, tol=1e-13, f=f)
        loss, g, _ = o2.gradient(th, rec, y)
        loss_ref += loss
        g_ref += g
    dev = torch.device("cuda", 0)
    mf = MultiFrequency.from_workloads(ws, batch_max=len(th), device=dev, maxit=3000)
    loss, grad, infos = mf.data_term_gradient(to_t(f, torch), to_t(th, torch), to_t(rec, torch),
                                              [to_t(y, torch) for y in ys])
    torch.cuda.synchronize()
    assert all(i["converged"] for fw, ad in infos for i in fw + ad)
    assert loss == pytest.approx(loss_ref, rel=1e-9)
    assert rel(grad.cpu().numpy(), g_ref) < 1e-8
    # the same handles, one at a time on the default stream
    seq = np.zeros_like(f)
    for i, w in enumerate(ws):
        s = Solver.from_workload(w, batch_max=len(th), device=dev, maxit=3000)
        s.set_contrast(to_t(f, torch))
        u, _ = s.forward(to_t(th, torch))
        _, G, _ = s.misfit(u, to_t(ys[i], torch), to_t(rec, torch))
        g, _ = s.gradient(to_t(th, torch), u, G)
        seq += g.cpu().numpy()
        s.close()
    assert rel(grad.cpu().numpy(), seq) < 1e-13
    mf.close()


def test_multifrequency_rejects_mixed_grids():
    torch = torch_cuda()
    from paper_2107_03679_gb300 import Solver
    from paper_2107_03679_gb300.multi import MultiFrequency
    a = W.small_workload(n_int=24, abl=4, levels=3)
    b = W.small_workload(n_int=32, abl=4, levels=3)
    dev = torch.device("cuda", 0)
    sa = Solver.from_workload(a, batch_max=1, device=dev)
    sb = Solver.from_workload(b, batch_max=1, device=dev)
    with pytest.raises(ValueError):
        MultiFrequency([sa, sb])
    sa.close()
    sb.close()
