"""Accelerated forward-backward splitting for the MAP problem of Sec. V (Alg. 4), on the GPU.

    f* = argmin_{f >= 0} sum_q 1/2 ||S u_sc,q(f) - y_q||^2 + tau TV(f)

Every iteration runs the forward solves of its angles (mgh_forward), the data term and its
adjoint source (mgh_misfit), the adjoint solves and the gradient (mgh_gradient, Prop. 1), the
backward step prox_{gamma tau}(fbar - gamma d) (mgh_tv_prox: nonnegativity + isotropic TV by fast
gradient projection on the dual) and the momentum step (mgh_fbs_momentum).  The angles of an
iteration are given by the caller: a random subset of the illuminations (the stochastic variant of
Alg. 4) or all of them.  This module only orders the library calls and keeps the buffers.
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Sequence

import torch

from .solver import Solver


def fbs(solver: Solver, theta: torch.Tensor, rec: torch.Tensor, y: torch.Tensor, f0: torch.Tensor,
        subsets: Sequence, gamma: float, tau: float, prox_iters: int = 100,
        callback: Optional[Callable[[int, torch.Tensor, float], None]] = None):
    """Alg. 4 from f0: fbar^1 = f^0, alpha_1 = 1; for each entry of `subsets` (angle indices),
        d    = sum over those angles of the data-term gradient at fbar
        f    = prox_{gamma tau}(fbar - gamma d)
        alpha' = (1 + sqrt(1 + 4 alpha^2)) / 2,   fbar = f + (alpha - 1) / alpha' (f - f_prev).
    theta: [Q] angles, y: [Q][M] measurements at the receivers rec; f0: [ny_int][nx_int].
    Returns (f, losses, infos): the last iterate, the data term at each fbar, and the solve
    records of each iteration (forward, adjoint)."""
    dev = solver.device
    theta = theta.to(device=dev, dtype=torch.float64).reshape(-1).contiguous()
    y = y.to(device=dev, dtype=torch.complex128).contiguous()
    rec = rec.to(device=dev, dtype=torch.int64).contiguous()
    f_prev = f0.to(device=dev, dtype=torch.float64).clone().contiguous()
    f_bar = f_prev.clone()
    f_next = torch.empty_like(f_prev)
    alpha = 1.0
    losses: List[float] = []
    infos = []
    u = None
    for it, idx in enumerate(subsets):
        idx = torch.as_tensor(idx, dtype=torch.int64).to(dev)
        th = theta.index_select(0, idx)
        solver.set_contrast(f_bar)
        if u is None or u.shape[0] != th.numel():
            u = solver.field(th.numel())
        u, inf_f = solver.forward(th, out=u)
        _, G, loss = solver.misfit(u, y.index_select(0, idx), rec)
        d, inf_a = solver.gradient(th, u, G)
        solver.tv_prox(f_bar, d, gamma, gamma * tau, prox_iters, out=f_next)
        alpha_n = (1.0 + math.sqrt(1.0 + 4.0 * alpha * alpha)) / 2.0
        solver.fbs_momentum(f_next, f_prev, (alpha - 1.0) / alpha_n, out=f_bar)
        f_prev, f_next = f_next, f_prev
        alpha = alpha_n
        losses.append(loss)
        infos.append((inf_f, inf_a))
        if callback is not None:
            callback(it, f_prev, loss)
    return f_prev, losses, infos


def snr_db(eta: torch.Tensor, eta_true: torch.Tensor) -> float:
    """20 log10(||eta_true|| / ||eta_true - eta||) (Sec. VI), of two device fields."""
    num = torch.linalg.vector_norm(eta_true)
    den = torch.linalg.vector_norm(eta_true - eta)
    return float(20.0 * torch.log10(num / den))
