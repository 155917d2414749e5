"""The s-step operator product v_{k+1} = A z_k formed by the level-0 post-smoothing kernel itself
(k_post_waf) against the separate product kernel (MGH_FUSE_MATVEC=0).

The fused kernel forms every entry of v_{k+1} with the separate kernel's operations on the same
stored z_k; only the order in which ||v_{k+1}||^2 is summed
differs (per row pair and strip, then in FP64).  Both solves must meet the oracle's exact solution, with
step counts within two of each other, and the fused path must launch fewer kernels.  Grids: two
even widths, one with a ragged last strip; 1, 2 and 3 fine-level sweeps (each count has its own
kernel) with one sweep on the coarser levels.  Under FP16 storage the product stays in its own
kernel (faster there), so both runs must be the same."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _w(precision, n=120):
    return W.Workload("fuse", n, n - 18, 8, 8.0, 3, -40.0, 40.0, "ellipses", 5, levels=4, nu1=1, nu2=1,
                      restart=8, precision=precision, tol=1e-10)


@pytest.mark.parametrize("nu,precision,n", [(2, "mixed32", 120), (1, "mixed32", 98), (3, "mixed32", 120),
                                            (2, "mixed16", 120)])
def test_fused_product_matches_the_separate_kernel(nu, precision, n, monkeypatch):
    torch = torch_cuda()
    from paper_2107_03679_gb300 import capi
    w = _w(precision, n)
    p, f, o = oracle_solver(w)
    # nu sweeps on the fine level (the fused kernel's), one on the coarser levels
    nus = [nu, 1, 1]
    b = np.stack([O.rhs(p, f, t) for t in W.angles(w)])
    res = {}
    for fuse in ("1", "0"):
        monkeypatch.setenv("MGH_FUSE_MATVEC", fuse)
        s = make_solver(w, B=3, maxit=6000, arnoldi="sstep", nu1=nus, nu2=nus)
        s.set_contrast(torch.from_numpy(f).cuda())
        capi.mgh_launch_count(s._h, reset=True)
        x, infos = s.solve(torch.from_numpy(b).cuda())
        res[fuse] = (x.cpu().numpy(), [i["iterations"] for i in infos], capi.mgh_launch_count(s._h),
                     all(i["converged"] for i in infos))
        s.close()
    for fuse in ("1", "0"):
        x, its, _, conv = res[fuse]
        assert conv, (fuse, its)
        for q in range(3):
            assert rel(x[q], O.direct_solve(p, o.D, b[q])) < 1e-5
    assert all(abs(a - c) <= 2 for a, c in zip(res["1"][1], res["0"][1])), (res["1"][1], res["0"][1])
    if precision == "mixed16":
        # FP16 storage keeps the product in its own kernel: the same launches and the same solve
        assert res["1"][2] == res["0"][2]
        np.testing.assert_array_equal(res["1"][0], res["0"][0])
    else:
        # one product kernel fewer per step
        assert res["1"][2] <= res["0"][2] - min(res["1"][1]), (res["1"][2], res["0"][2])
