"""Host logic of the multi-rank path on CPU: 2 gloo ranks shard the angles, each computes its
share of the data-term gradient (with the FP64 oracle standing in for the per-rank GPU solve),
and one all-reduce gives the single-process gradient."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import workloads as W
from paper_2107_03679_gb300.distributed import shard, allreduce_sum_


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    w = W.Workload("mr", 12, 12, 3, 6.0, 5, -40.0, 40.0, "gt_ellipse", 4, levels=2, nu1=1, nu2=1,
                   precision="fp64")
    p = O.Problem.from_workload(w)
    f_gt = W.phantom(w)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    gt = O.MGHSolver(p, f_gt, levels=2, nu1=1, nu2=1, tol=1e-12)
    y = O.sample(gt.forward(th)[0], rec)
    return p, 0.5 * f_gt, th, rec, y


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, f, th, rec, y = _problem()
        a, b = shard(len(th), rank, world)
        s = O.MGHSolver(p, f, levels=2, nu1=1, nu2=1, tol=1e-12)
        loss, g, _ = s.gradient(th[a:b], rec, y[a:b])
        packed = torch.cat([torch.tensor([loss], dtype=torch.float64), torch.from_numpy(g).reshape(-1)])
        allreduce_sum_(packed)
        out[rank] = packed.numpy().copy()
    finally:
        dist.destroy_process_group()


def test_shard_covers_everything_once():
    for n in [0, 1, 5, 60, 61]:
        for world in [1, 2, 3, 8]:
            parts = [shard(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_sum_to_single_process_gradient():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    p, f, th, rec, y = _problem()
    s = O.MGHSolver(p, f, levels=2, nu1=1, nu2=1, tol=1e-12)
    loss, g, _ = s.gradient(th, rec, y)
    for r in range(world):
        assert out[r][0] == pytest.approx(loss, rel=1e-12)
        np.testing.assert_allclose(out[r][1:], g.reshape(-1), rtol=1e-10, atol=1e-14 * np.abs(g).max())


class _OracleStandIn:
    """CPU stand-in for the GPU Solver with the four calls sharded_loss_and_gradient makes
    (set_contrast, forward, misfit, gradient), backed by the FP64 oracle: the host logic of the
    multi-rank path runs unchanged on gloo ranks without a GPU."""

    def __init__(self, p):
        self.p = p
        self.s = None

    def set_contrast(self, f_d):
        self.s = O.MGHSolver(self.p, f_d.numpy(), levels=2, nu1=1, nu2=1, tol=1e-12)

    def forward(self, theta):
        u, infos = self.s.forward(theta.numpy())
        return torch.from_numpy(u), infos

    def misfit(self, u, y, rec):
        r, loss = O.misfit(O.sample(u.numpy(), rec.numpy()), y.numpy())
        G = np.zeros((u.shape[0], self.p.ny * self.p.nx), dtype=np.complex128)
        G[:, rec.numpy()] = r                      # G = S^T r, the adjoint source
        return torch.from_numpy(r), torch.from_numpy(G.reshape(u.shape)), loss

    def gradient(self, theta, u, G):
        g = np.zeros((self.p.ny_int, self.p.nx_int))
        for q, th in enumerate(theta.numpy()):
            z, _ = self.s.solve(np.conj(G[q].numpy()))           # A z_q = conj(G_q)
            u_tot = u[q].numpy() + O.incident_field(self.p, float(th))
            g += O.gradient_from_adjoint(self.p, z[None], u_tot[None])
        return torch.from_numpy(g), []


def _sharded_rank_main(rank, world, port, out):
    from paper_2107_03679_gb300.distributed import sharded_loss_and_gradient
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, f, th, rec, y = _problem()
        loss, g = sharded_loss_and_gradient(_OracleStandIn(p), torch.from_numpy(f), torch.from_numpy(th),
                                            torch.from_numpy(rec), torch.from_numpy(y), rank, world)
        out[rank] = np.concatenate([[loss], g.numpy().reshape(-1)])
    finally:
        dist.destroy_process_group()


def test_sharded_loss_and_gradient_on_two_gloo_ranks():
    """distributed.sharded_loss_and_gradient itself: each of 2 gloo ranks solves its share of the
    5 angles (3 + 2) through the solver interface, one all-reduce sums (loss, gradient), and every
    rank ends with the single-process loss and gradient."""
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_sharded_rank_main, args=(world, port, out), nprocs=world, join=True)
    p, f, th, rec, y = _problem()
    s = O.MGHSolver(p, f, levels=2, nu1=1, nu2=1, tol=1e-12)
    loss, g, _ = s.gradient(th, rec, y)
    for r in range(world):
        assert out[r][0] == pytest.approx(loss, rel=1e-12)
        np.testing.assert_allclose(out[r][1:], g.reshape(-1), rtol=1e-10, atol=1e-14 * np.abs(g).max())
