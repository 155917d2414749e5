"""Host-side logic of the package, on the CPU: solver parameters (cycle type, per-level sweeps)
validated by the library's own host check; the order of calls and the buffers of the FBS driver
(Alg. 4), run against a fake solver whose steps are the oracle's; the threads of the concurrent
multi-handle driver (results in order, the first exception re-raised); the multi-frequency
workloads."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
import paper_2107_03679_gb300.capi as capi
from paper_2107_03679_gb300.solver import make_params
from paper_2107_03679_gb300.reconstruct import fbs


def test_make_params_uniform_and_per_level_sweeps():
    p, arnoldi = make_params(128, 128, 16, 1.0, 2 * math.pi / 10, levels=4, nu1=2, nu2=1, restart=8)
    assert arnoldi == "sstep" and p.nu_per_level == 0 and (p.nu1, p.nu2) == (2, 1)
    assert capi.mgh_workspace_bytes(p) > 0
    p, _ = make_params(128, 128, 16, 1.0, 2 * math.pi / 10, levels=4, nu1=np.array([2, 1, 0]),
                       nu2=[0, 1, 2], cycle_type="w", precision="fp64")
    assert p.nu_per_level == 1 and list(p.nu1_level)[:3] == [2, 1, 0] and list(p.nu2_level)[:3] == [0, 1, 2]
    assert p.cycle_type == 2 and p.precision == capi.MGH_PREC_FP64
    assert capi.mgh_workspace_bytes(p) > 0
    with pytest.raises(ValueError):
        make_params(128, 128, 16, 1.0, 0.6, levels=4, nu1=[2, 1], nu2=2)
    bad, _ = make_params(128, 128, 16, 1.0, 0.6, levels=4, nu1=[2, 5, 1], nu2=2)
    with pytest.raises(capi.MGHError):
        capi.mgh_workspace_bytes(bad)


class FakeSolver:
    """The calls fbs() makes, on CPU tensors: per angle q the data term 1/2 ||f - C_q||^2 (C_q is
    the real part of y[q]), the TV prox of the oracle and the momentum step written out."""

    def __init__(self, shape):
        self.device = torch.device("cpu")
        self.shape = shape
        self.f = None
        self.calls = []

    def set_contrast(self, f):
        self.f = f.clone()
        self.calls.append("set_contrast")

    def field(self, B):
        return torch.zeros((B, 1), dtype=torch.complex128)

    def forward(self, th, out=None):
        self.calls.append("forward")
        return out, [dict(iterations=1, converged=True)] * th.numel()

    def misfit(self, u, y, rec):
        self.calls.append("misfit")
        self.C = [y[q].real.reshape(self.shape) for q in range(y.shape[0])]
        loss = sum(0.5 * float(torch.sum((self.f - c) ** 2)) for c in self.C)
        return None, None, loss

    def gradient(self, th, u, G):
        self.calls.append("gradient")
        return sum(self.f - c for c in self.C), [dict(iterations=1, converged=True)] * th.numel()

    def tv_prox(self, fbar, d, gamma, lam, iters, out=None):
        self.calls.append("tv_prox")
        out[:] = torch.from_numpy(O.tv_prox((fbar - gamma * d).numpy(), lam, iters))
        return out

    def fbs_momentum(self, f, f_prev, c, out=None):
        self.calls.append("fbs_momentum")
        out[:] = f + c * (f - f_prev)
        return out


def test_fbs_driver_follows_the_oracle_recursion():
    shape = (7, 9)
    rng = np.random.default_rng(3)
    C = rng.uniform(-0.2, 0.6, size=(5,) + shape)
    y = torch.from_numpy(C.reshape(5, -1).astype(np.complex128))
    subsets = W.angle_subsets(5, 2, 6, seed=8)
    gamma, tau, iters = 0.3, 0.05, 30
    ref_losses = []

    def grad_fn(f, idx):
        ref_losses.append(sum(0.5 * float(np.sum((f - C[q]) ** 2)) for q in idx))
        return sum(f - C[q] for q in idx)

    ref = O.fbs(grad_fn, np.zeros(shape), subsets, gamma, tau, prox_iters=iters)
    s = FakeSolver(shape)
    seen = []
    f, losses, infos = fbs(s, torch.arange(5, dtype=torch.float64), torch.zeros(1, dtype=torch.int64), y,
                           torch.zeros(shape, dtype=torch.float64), subsets, gamma, tau, prox_iters=iters,
                           callback=lambda it, fk, loss: seen.append(fk.clone()))
    np.testing.assert_allclose(f.numpy(), ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose(losses, ref_losses, rtol=1e-14)
    assert len(infos) == len(subsets) and len(seen) == len(subsets)
    assert torch.equal(seen[-1], f)
    assert s.calls[:6] == ["set_contrast", "forward", "misfit", "gradient", "tv_prox", "fbs_momentum"]
    assert float(f.min()) >= 0.0


def test_run_concurrently_orders_results_and_reraises():
    import threading
    from paper_2107_03679_gb300.multi import run_concurrently

    class Job:
        stream = None

        def __init__(self, k):
            self.k = k

    seen = set()
    barrier = threading.Barrier(4, timeout=10)

    def fn(i, job):
        barrier.wait()            # all four run at the same time, each in its own thread
        seen.add(threading.get_ident())
        return job.k * 10 + i

    assert run_concurrently([Job(k) for k in range(4)], fn) == [0, 11, 22, 33]
    assert len(seen) == 4

    def bad(i, job):
        if i == 2:
            raise RuntimeError("frequency 2 failed")
        return i

    with pytest.raises(RuntimeError, match="frequency 2"):
        run_concurrently([Job(k) for k in range(3)], bad)


def test_multifrequency_workloads_scale_points_per_wavelength():
    base = W.WORKLOADS["ellipses576"]
    ws = W.multifrequency_workloads(base)
    assert [round(w.ppw, 3) for w in ws] == [26.667, 16.0, 13.333, 10.0]
    assert all(w.nx == base.nx and w.seed == base.seed and w.n_angles == base.n_angles for w in ws)
    assert np.array_equal(W.phantom(ws[0]), W.phantom(base))
    assert ws[-1].k == pytest.approx(base.k) and ws[0].k == pytest.approx(base.k * 3 / 8)


class _OracleStandIn:
    """CPU stand-in for a Solver handle (the calls SplitBatch makes), backed by the FP64 oracle."""

    stream = None

    def __init__(self, p, levels=2):
        self.p, self.levels, self.s = p, levels, None

    def set_contrast(self, f_d):
        self.s = O.MGHSolver(self.p, f_d.numpy(), levels=self.levels, nu1=1, nu2=1, tol=1e-12)

    def forward(self, theta, out=None):
        u, infos = self.s.forward(theta.numpy())
        out.copy_(torch.from_numpy(u))
        return out, infos

    def crop(self, u):
        return torch.from_numpy(O.crop(self.p, u.numpy()))

    def misfit(self, u, y, rec):
        r, loss = O.misfit(O.sample(u.numpy(), rec.numpy()), y.numpy())
        G = np.zeros((u.shape[0], self.p.ny * self.p.nx), dtype=np.complex128)
        G[:, rec.numpy()] = r
        return torch.from_numpy(r), torch.from_numpy(G.reshape(u.shape)), loss

    def gradient(self, theta, u, G):
        g = np.zeros((self.p.ny_int, self.p.nx_int))
        infos = []
        for q, th in enumerate(theta.numpy()):
            z, info = self.s.solve(np.conj(G[q].numpy()))
            infos.append(info)
            g += O.gradient_from_adjoint(self.p, z[None], (u[q].numpy() + O.incident_field(self.p, float(th)))[None])
        return torch.from_numpy(g), infos


def test_split_batch_equals_one_handle_over_all_angles():
    """SplitBatch: 5 angles over 2 parts (3 + 2), each part solving its share in its own thread;
    loss, gradient, fields, cropped fields and infos equal one solver's over all angles."""
    from paper_2107_03679_gb300.multi import SplitBatch
    w = W.Workload("split", 12, 12, 3, 6.0, 5, -40.0, 40.0, "gt_ellipse", 4, levels=2, nu1=1, nu2=1,
                   precision="fp64")
    p = O.Problem.from_workload(w)
    f_gt = W.phantom(w)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    gt = O.MGHSolver(p, f_gt, levels=2, nu1=1, nu2=1, tol=1e-12)
    y = O.sample(gt.forward(th)[0], rec)
    f = 0.5 * f_gt
    sb = SplitBatch([_OracleStandIn(p), _OracleStandIn(p)])
    assert sb.ranges(5) == [(0, 3), (3, 5)]
    u = torch.zeros((5, p.ny, p.nx), dtype=torch.complex128)
    uc = torch.zeros((5, p.ny_int, p.nx_int), dtype=torch.complex128)
    loss, g, inf_f, inf_a = sb.data_term_gradient(torch.from_numpy(f), torch.from_numpy(th), torch.from_numpy(rec),
                                                  torch.from_numpy(y), u, crop_out=uc)
    ref = O.MGHSolver(p, f, levels=2, nu1=1, nu2=1, tol=1e-12)
    loss_ref, g_ref, u_ref = ref.gradient(th, rec, y)
    assert loss == pytest.approx(loss_ref, rel=1e-12)
    np.testing.assert_allclose(g.numpy(), g_ref, rtol=1e-10, atol=1e-14 * np.abs(g_ref).max())
    np.testing.assert_allclose(u.numpy(), u_ref, rtol=0, atol=1e-12 * np.abs(u_ref).max())
    np.testing.assert_array_equal(uc.numpy(), O.crop(p, u.numpy()))
    assert len(inf_f) == 5 and len(inf_a) == 5


def test_bench_byte_model_with_and_without_the_fused_product():
    """The bench's algorithmic bytes for the s-step engine: with the basis product in its own kernel
    it reads z and writes v_{k+1} (16 B per point and step plus D_A per launch); fused into the
    level-0 post kernel, the post class carries the v_{k+1} write and D_A instead and there is no
    product class.  The captured ncu traffic is reported only for the kernel that was captured."""
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    N, cs = 1000, 8
    prof = {"arnoldi_steps": 40, "cycle_steps": 48, "gram_reads": 54, "residuals": 7, "updates": 6,
            "update_reads": 40}
    sep = {"vcycle_pre_l0": 48, "vcycle_post_l0": 48, "matvec_dots": 48}
    fus = {"vcycle_pre_l0": 48, "vcycle_post_l0": 48, "matvec_dots": 0}
    a = bench.algorithmic_bytes(prof, N, cs, sep, "sstep")
    b = bench.algorithmic_bytes(prof, N, cs, fus, "sstep")
    assert a["matvec_dots"] == 48 * N * (cs + cs) + 48 * cs * N
    assert "matvec_dots" not in b
    # fused: the post class gains the v_{k+1} write and D_A, not the z re-read
    assert b["vcycle_post_l0"] - a["vcycle_post_l0"] == 48 * N * cs + 48 * cs * N
    assert sum(a.values()) - sum(b.values()) == 48 * N * cs   # the z re-read saved
    w = W.WORKLOADS["ellipses576"]
    fused_cap = bench.captured_traffic("vcycle_post_l0", w, "mixed32", 60, fused=True)
    assert (fused_cap is not None) == bench.POST_CAPTURE_FUSED
    assert (bench.captured_traffic("vcycle_post_l0", w, "mixed32", 60, fused=False) is None) == bench.POST_CAPTURE_FUSED
    if fused_cap is not None:
        cap, once = bench.NCU_TRAFFIC_24["vcycle_post_l0"]
        assert fused_cap == round((cap - once) * 60 / 24 + once)
    assert bench.captured_traffic("vcycle_post_l0", w, "mixed32", 60, shape={"wave_warps": 2}) is None


def test_bench_byte_model_of_idrs():
    """The bench's algorithmic bytes for IDR(s), counted by hand for one outer step of s = 1 (two
    cycles, FP32 cycle input and output, cs = 8): the intermediate step reads r and G_0 and writes
    v (40 B), reads U_0 and y and writes U_0 (40 B), then updates G_0, U_0, r, x (read 4 x 16, write
    4 x 16: 128 B); the dimension reduction reads y, x, r, t and writes x, r (88 B).  The products
    G_0 = A U_0 (32 B) and t = A y (cs + 32 B) carry D_A per launch."""
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    N, cs = 1000, 8
    prof = {"arnoldi_steps": 20, "residuals": 3}
    launches = {"vcycle_pre_l0": 20, "vcycle_post_l0": 20, "matvec_dots": 20}
    a = bench.algorithmic_bytes(prof, N, cs, launches, "idrs", idr_s=1)
    outer = 20 / 2
    assert a["gs_update"] == outer * N * (40 + 40 + 128 + 88)
    assert a["matvec_dots"] == outer * N * (32 + cs + 32) + 20 * 16 * N
    b = bench.algorithmic_bytes(prof, N, cs, launches, "bicgstab")
    for k in ("vcycle_pre_l0", "vcycle_post_l0", "true_residual"):      # the same cycle and check
        assert a[k] == b[k]
    # larger s: more vector bytes per cycle (the U and G combinations grow with s)
    per_cycle = [bench.algorithmic_bytes(prof, N, cs, launches, "idrs", idr_s=s)["gs_update"] for s in (1, 2, 4, 8)]
    assert all(x < y for x, y in zip(per_cycle, per_cycle[1:]))
