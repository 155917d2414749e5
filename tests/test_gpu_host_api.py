"""The host-buffer entry point mgh_data_term_gradient_host: contrast, angles, receivers and data
from host memory, loss, gradient and receiver residuals back to host memory, in one call.  It runs
the device-pointer sequence (mgh_set_contrast, mgh_forward, mgh_misfit, mgh_gradient) on the
handle's staging buffers, so its results equal those calls' bit for bit, and they meet the
oracle's gradient within the mixed tolerance."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def test_host_buffer_call_equals_device_calls_and_oracle():
    torch = torch_cuda()
    w = W.Workload("hostapi", 70, 53, 9, 8.0, 4, -50.0, 40.0, "gt_ellipse", 4, levels=4, nu1=2, nu2=2,
                   restart=8, precision="mixed32", tol=1e-10)
    p, f_gt, o = oracle_solver(w, tol=1e-13)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    y = O.sample(o.forward(th)[0], rec) + W.complex_noise((len(th), rec.size), 0.01, 4)
    f = 0.6 * f_gt
    s = make_solver(w, B=len(th), maxit=6000)
    # device-pointer calls
    d_th, d_rec, d_y = (torch.from_numpy(a).cuda() for a in (th, rec, y))
    s.set_contrast(torch.from_numpy(f).cuda())
    u, _ = s.forward(d_th)
    r_dev, G, loss_dev = s.misfit(u, d_y, d_rec)
    g_dev, _ = s.gradient(d_th, u, G)
    # one host-buffer call, pinned and pageable inputs
    for pin in (True, False):
        h = [torch.from_numpy(np.ascontiguousarray(a)) for a in (f, th, rec, y)]
        if pin:
            h = [t.pin_memory() for t in h]
        loss, g, r, inf_f, inf_a = s.data_term_gradient_host(*h, want_infos=True)
        assert all(i["converged"] for i in inf_f + inf_a)
        assert loss == loss_dev
        np.testing.assert_array_equal(g.numpy(), g_dev.cpu().numpy())
        np.testing.assert_array_equal(r.numpy(), r_dev.cpu().numpy())
    _, _, o2 = oracle_solver(w, tol=1e-13, f=f)
    loss_ref, g_ref, _ = o2.gradient(th, rec, y)
    assert loss == pytest.approx(loss_ref, rel=1e-8)
    assert rel(g.numpy(), g_ref) < 1e-5
    from paper_2107_03679_gb300 import capi
    with pytest.raises(ValueError):            # device tensors are refused by the host-buffer binding
        s.data_term_gradient_host(torch.from_numpy(f).cuda(), *h[1:])
    s.close()
