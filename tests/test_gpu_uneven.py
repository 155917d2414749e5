"""The uneven batch (grids of different sizes, each with its own angles, solved together on
concurrent streams): every grid's fields meet the oracle's exact discrete solution, one grid on
the plain FP64 path and the others mixed, and equal what each handle gives when run alone."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _grids():
    # 48^2, 64^2 and 80^2 interiors (layer n/16 = 3..5 cells), 8 points per wavelength, 3, 2 and 4 angles
    spec = [(48, 3, 3, 61, "mixed32"), (64, 2, 3, 62, "fp64"), (80, 4, 4, 63, "mixed32")]
    return [W.Workload(f"uneven{n}", n, n, n // 16, 8.0, b, -50.0, 50.0, "ellipses", seed, levels=lv, nu1=1,
                       nu2=1, restart=8, precision=prec, tol=1e-10 if prec == "mixed32" else 1e-12)
            for n, b, lv, seed, prec in spec]


def test_uneven_batch_fields_match_direct_solves_and_solo_runs():
    torch = torch_cuda()
    from paper_2107_03679_gb300.multi import UnevenBatch
    ws = _grids()
    dev = torch.device("cuda", 0)
    ub = UnevenBatch.from_workloads(ws, device=dev, maxit=6000)
    fs = [torch.from_numpy(W.phantom(w)).to(dev) for w in ws]
    ths = [torch.from_numpy(W.angles(w)).to(dev) for w in ws]
    res = ub.forward(fs, ths)
    torch.cuda.synchronize()
    for w, (u, infos) in zip(ws, res):
        p, f, o = oracle_solver(w)
        u = u.cpu().numpy()
        bound = 1e-5 if w.precision == "mixed32" else 1e-10
        for q, t in enumerate(W.angles(w)):
            assert infos[q]["converged"], (w.name, infos)
            assert rel(u[q], O.direct_solve(p, o.D, O.rhs(p, f, t))) < bound, w.name
    # each grid alone on its own handle: the same fields (same handle configuration and arithmetic)
    for i, w in enumerate(ws):
        s = ub.solvers[i]
        s.set_contrast(fs[i])
        u, _ = s.forward(ths[i])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(u.cpu().numpy(), res[i][0].cpu().numpy())
    ub.close()
