"""Launch shapes of the FP32 level kernels (mgh_set_kernel_shape) and the autotuner that picks them.

A shape changes the schedule, never the arithmetic of a point: the wavefront kernels recompute
their halo rows with the same operations whatever the segment length, warps per block or ring
depth, so the solve is bit-identical; so does splitting the coarse tail of a right-hand side over a
cluster of blocks.  Moving the first level of the one-kernel coarse tail swaps
level kernels for the tail kernel on some levels (same cycle, other rounding order), so the solve
still meets the direct solution within the mixed tolerance."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _w():
    # 136 x 118: three wavefront strips, a ragged last one; levels 136, 68, 34, 17: the tail starts at level 1 or 2
    return W.Workload("shape", 120, 102, 8, 8.0, 3, -40.0, 40.0, "ellipses", 5, levels=4, nu1=1, nu2=1,
                      restart=8, precision="mixed32", tol=1e-10)


def test_kernel_shapes_leave_the_solve_unchanged():
    torch = torch_cuda()
    from paper_2107_03679_gb300 import capi
    w = _w()
    p, f, o = oracle_solver(w)
    b = np.stack([O.rhs(p, f, t) for t in W.angles(w)])
    s = make_solver(w, B=3, maxit=6000)
    s.set_contrast(torch.from_numpy(f).cuda())
    base = s.kernel_shape()
    assert base["wave_seg"] == [0] * 12 and base["wave_warps"] == 4 and base["wave_ring"] == 1 and base["tail_level"] >= 1
    x0, inf0 = s.solve(torch.from_numpy(b).cuda())
    x0 = x0.cpu().numpy()
    for shape in (dict(wave_seg=16), dict(wave_seg=[64, 24, 8], wave_warps=2), dict(wave_ring=2), dict(wave_seg=6),
                  dict(tail_cluster=2), dict(tail_cluster=4)):
        s.set_kernel_shape(**dict(base, **shape))
        x, inf = s.solve(torch.from_numpy(b).cuda())
        np.testing.assert_array_equal(x.cpu().numpy(), x0)
        assert [i["iterations"] for i in inf] == [i["iterations"] for i in inf0]
    for tail in (0, base["tail_level"] + 1):
        s.set_kernel_shape(**dict(base, tail_level=tail))
        assert s.kernel_shape()["tail_level"] == tail
        x, inf = s.solve(torch.from_numpy(b).cuda())
        for q in range(3):
            assert inf[q]["converged"] and rel(x.cpu().numpy()[q], O.direct_solve(p, o.D, b[q])) < 1e-5
    for bad in (dict(wave_warps=3), dict(wave_ring=3), dict(tail_level=3), dict(wave_seg=[0, -1]), dict(tail_cluster=3),
                dict(tail_level=0, tail_cluster=2)):
        with pytest.raises(capi.MGHError):
            s.set_kernel_shape(**dict(base, **bad))
    s.close()


def test_autotuner_returns_a_valid_shape_and_caches_it(tmp_path, monkeypatch):
    torch = torch_cuda()
    import paper_2107_03679_gb300.autotune as A
    monkeypatch.setattr(A, "CACHE", str(tmp_path / "tune.json"))
    w = _w()
    f = torch.from_numpy(W.phantom(w)).cuda()
    th = torch.from_numpy(W.angles(w)).cuda()
    shape, trials = A.tune_shapes(w, f, th, torch.device("cuda", 0), steps=16)
    assert len(trials) >= 5 and shape["ms_per_step"] <= shape["builtin_ms_per_step"]
    assert shape["wave_warps"] in (2, 4) and shape["wave_ring"] in (1, 2) and shape["tail_level"] >= 0
    again, trials2 = A.tune_shapes(w, f, th, torch.device("cuda", 0), steps=16)
    assert trials2 == [] and again == shape
