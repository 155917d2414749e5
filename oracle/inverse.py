"""Reconstruction loop of Sec. V (oracle, test infrastructure).

* tv_prox: the proximal operator of the nonnegativity constraint plus isotropic total variation,
  prox_lam(w) = argmin_{x >= 0} 1/2 ||x - w||^2 + lam TV(x), computed by fast gradient projection
  on its dual (Beck & Teboulle 2009, constrained TV denoising), the solver named in Sec. V.
  TV(x) = sum_ij sqrt((x_ij - x_i+1,j)^2 + (x_ij - x_i,j+1)^2) with forward differences that
  are 0 across the last row / column.
* fbs: the accelerated forward-backward splitting of Alg. 4 (Beck & Teboulle 2009; Nesterov
  2013) on sum_q 1/2 ||S u_sc,q(f) - y_q||^2 + tau TV(f), f >= 0, with the angles of each
  iteration given (a random subset: the stochastic variant of Alg. 4) and a fixed step.
* snr: 20 log10(||eta_true|| / ||eta_true - eta||) dB on the refractive index (Sec. VI).
"""
from __future__ import annotations

from typing import Callable, List, Optional

import numpy as np


def grad_fwd(x: np.ndarray):
    """(dx_i, dx_j): forward differences x - x[shifted], 0 across the last row / column."""
    p = np.zeros_like(x)
    q = np.zeros_like(x)
    p[:-1, :] = x[:-1, :] - x[1:, :]
    q[:, :-1] = x[:, :-1] - x[:, 1:]
    return p, q


def grad_adj(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """The adjoint of grad_fwd: <grad_fwd x, (p, q)> = <x, grad_adj(p, q)> (the last row of p
    and the last column of q meet the zero differences and do not contribute)."""
    out = np.zeros_like(p)
    out[:-1, :] += p[:-1, :]
    out[1:, :] -= p[:-1, :]
    out[:, :-1] += q[:, :-1]
    out[:, 1:] -= q[:, :-1]
    return out


def tv(x: np.ndarray) -> float:
    p, q = grad_fwd(x)
    return float(np.sum(np.sqrt(p * p + q * q)))


def tv_prox(w: np.ndarray, lam: float, iters: int) -> np.ndarray:
    """argmin_{x >= 0} 1/2 ||x - w||^2 + lam TV(x) by fast gradient projection on the dual.

    With x(g) = max(0, w - lam grad_adj(g)) for a dual field g = (p, q), |g_ij| <= 1, the dual is
    maximised by projected gradient steps of size 1 / (8 lam) (8 bounds ||grad_fwd||^2) with
    Nesterov momentum; the primal solution is x(g) at the last dual iterate.
    """
    if lam <= 0.0:
        return np.maximum(w, 0.0)
    pr = np.zeros_like(w)
    qr = np.zeros_like(w)          # momentum point
    pp = np.zeros_like(w)
    qq = np.zeros_like(w)          # previous dual iterate
    t = 1.0
    for _ in range(iters):
        x = np.maximum(w - lam * grad_adj(pr, qr), 0.0)
        gp, gq = grad_fwd(x)
        pn = pr + gp / (8.0 * lam)
        qn = qr + gq / (8.0 * lam)
        nrm = np.maximum(1.0, np.sqrt(pn * pn + qn * qn))
        pn /= nrm
        qn /= nrm
        tn = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        c = (t - 1.0) / tn
        pr = pn + c * (pn - pp)
        qr = qn + c * (qn - qq)
        pp, qq, t = pn, qn, tn
    return np.maximum(w - lam * grad_adj(pp, qq), 0.0)


def snr(eta: np.ndarray, eta_true: np.ndarray) -> float:
    return float(20.0 * np.log10(np.linalg.norm(eta_true) / np.linalg.norm(eta_true - eta)))


def fbs(grad_fn: Callable[[np.ndarray, np.ndarray], np.ndarray], f0: np.ndarray, subsets: List[np.ndarray],
        gamma: float, tau: float, prox_iters: int = 100,
        callback: Optional[Callable[[int, np.ndarray], None]] = None) -> np.ndarray:
    """Alg. 4: f_bar^1 = f^0, alpha_1 = 1; iteration nu uses the angles subsets[nu] (drawn by the
    caller: the stochastic variant of Alg. 4, or every angle), d = the sum of their data-term
    gradients at f_bar (grad_fn(f_bar, angle_indices)), f = prox(f_bar - gamma d) with weight
    gamma tau, alpha' = (1 + sqrt(1 + 4 alpha^2)) / 2 and f_bar = f + (alpha - 1) / alpha' (f - f_prev)."""
    f_prev = f0.copy()
    f_bar = f0.copy()
    alpha = 1.0
    f = f0.copy()
    for it, idx in enumerate(subsets):
        d = grad_fn(f_bar, idx)
        f = tv_prox(f_bar - gamma * d, gamma * tau, prox_iters)
        alpha_n = (1.0 + np.sqrt(1.0 + 4.0 * alpha * alpha)) / 2.0
        f_bar = f + ((alpha - 1.0) / alpha_n) * (f - f_prev)
        f_prev, alpha = f, alpha_n
        if callback is not None:
            callback(it, f)
    return f
