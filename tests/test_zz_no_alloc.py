"""The allocation-free misfit entry point matches mgh_misfit.

mgh_misfit_noalloc serves callers that cannot allocate device memory (their memory belongs to a
pool they do not own, or they may not call cudaMalloc because it can synchronise the device):
it needs no handle and keeps its scratch in a static device array of the library.  Two calls in
a row, the second with a smaller batch and different data, must both agree with mgh_misfit, so a
stale scratch entry from the first call cannot leak into the second.  This file is collected
last on purpose.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_misfit_noalloc_matches_misfit_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_03679_gb300 import Solver, capi

    w = W.Workload("noalloc", 40, 30, 5, 8.0, 4, -30.0, 30.0, "ellipses", 17, levels=3, nu1=1, nu2=1,
                   precision="fp64")
    dev = torch.device("cuda", 0)
    s = Solver.from_workload(w, batch_max=4, device=dev)
    f = W.phantom(w)
    rec_np = W.receivers(w, f)
    rec = torch.from_numpy(rec_np).to(dev)
    M = rec.numel()
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call, (B, seed) in enumerate([(4, 1), (2, 2)]):
        u = torch.from_numpy(W.random_field((B, w.ny, w.nx), seed)).to(dev)
        y = torch.from_numpy(W.random_field((B, M), seed + 10)).to(dev)
        r_ref, G_ref, loss_ref = s.misfit(u, y, rec)
        r = torch.full((B, M), complex(7.0, 7.0), dtype=torch.complex128, device=dev)
        G = torch.full((B, w.ny, w.nx), complex(7.0, 7.0), dtype=torch.complex128, device=dev)
        loss = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        capi.mgh_misfit_noalloc(w.nx, w.ny, capi._ptr(u), capi._ptr(y), B, capi._ptr(rec), M, capi._ptr(r),
                                capi._ptr(G), capi._ptr(loss), stream)
        torch.cuda.synchronize()
        assert torch.equal(r, r_ref), call
        assert torch.equal(G, G_ref), call
        assert float(loss.item()) == pytest.approx(loss_ref, rel=1e-13, abs=0.0), call
    too_big = 4097
    with pytest.raises(capi.MGHError):
        capi.mgh_misfit_noalloc(w.nx, w.ny, capi._ptr(u), capi._ptr(y), too_big, capi._ptr(rec), M,
                                capi._ptr(r), capi._ptr(G), capi._ptr(loss), stream)
    s.close()
