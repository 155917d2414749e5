"""Parity of the reconstruction loop (Sec. V, Alg. 4) on the GPU with the FP64 oracle.

* mgh_tv_prox against oracle.tv_prox with the same iteration count: both run the same FP64
  recursion, so they agree to rounding (relative L2 <= 1e-12), on a 70 x 53 interior (ragged
  against the 256-thread blocks), with and without the gradient move, for lam = 0 (the clamp),
  and with the output aliasing the input.
* mgh_fbs_momentum against its formula (1e-15).
* Four accelerated FBS iterations on stochastic angle subsets (the GPU driver against
  oracle.fbs fed by the oracle's data-term gradient): each side solves to a residual of 1e-12,
  the gradients then agree to ~1e-9 and the iterates to 1e-8.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def to_t(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ragged():
    return W.Workload("ragged", 70, 53, 9, 8.0, 2, -50.0, 40.0, "ellipses", 11, levels=4, nu1=1, nu2=1,
                      precision="fp64")


def _real_field(w, seed, shift=0.0, scale=1.0):
    return scale * np.real(W.random_field((w.ny_int, w.nx_int), seed)) + shift


@pytest.mark.parametrize("lam", [0.0, 0.05, 0.4])
@pytest.mark.parametrize("iters", [1, 6, 100])
def test_tv_prox_matches_oracle(lam, iters):
    torch = torch_cuda()
    w = _ragged()
    s = make_solver(w, B=2)
    fbar = _real_field(w, 31, shift=0.3)
    d = _real_field(w, 32)
    gamma = 0.7
    ref = O.tv_prox(fbar - gamma * d, lam, iters)
    out = s.tv_prox(to_t(fbar, torch), to_t(d, torch), gamma, lam, iters).cpu().numpy()
    assert rel(out, ref) < 1e-12
    assert out.min() >= 0.0
    # without the gradient move, writing over the input
    buf = to_t(fbar, torch)
    s.tv_prox(buf, None, gamma, lam, iters, out=buf)
    assert rel(buf.cpu().numpy(), O.tv_prox(fbar, lam, iters)) < 1e-12


def test_tv_prox_reduces_the_objective_and_is_idempotent_on_constants():
    torch = torch_cuda()
    w = _ragged()
    s = make_solver(w, B=2)
    wf = _real_field(w, 33, shift=0.5)
    lam = 0.2
    x = s.tv_prox(to_t(wf, torch), None, 0.0, lam, 200).cpu().numpy()
    obj = lambda z: 0.5 * np.sum((z - wf) ** 2) + lam * O.tv(z)
    assert obj(x) < obj(np.maximum(wf, 0.0))
    const = np.full((w.ny_int, w.nx_int), 0.25)
    xc = s.tv_prox(to_t(const, torch), None, 0.0, lam, 20).cpu().numpy()
    assert np.max(np.abs(xc - const)) < 1e-14


def test_fbs_momentum():
    torch = torch_cuda()
    w = _ragged()
    s = make_solver(w, B=2)
    f, fp = _real_field(w, 34), _real_field(w, 35)
    c = 0.37
    out = s.fbs_momentum(to_t(f, torch), to_t(fp, torch), c).cpu().numpy()
    assert rel(out, f + c * (f - fp)) < 1e-15
    # fbar may alias f_prev
    buf = to_t(fp, torch)
    s.fbs_momentum(to_t(f, torch), buf, c, out=buf)
    assert rel(buf.cpu().numpy(), f + c * (f - fp)) < 1e-15


def test_fbs_iterations_match_oracle():
    torch = torch_cuda()
    from paper_2107_03679_gb300.reconstruct import fbs
    w = W.Workload("fbssmall", 24, 20, 6, 8.0, 4, -40.0, 40.0, "gt_ellipse", 4, levels=3, nu1=1, nu2=1,
                   precision="fp64", tol=1e-12)
    p, f_gt, o = oracle_solver(w, tol=1e-13)
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    u, _ = o.forward(th)
    y = O.sample(u, rec) + W.complex_noise((len(th), rec.size), 0.01, 6)
    subsets = W.angle_subsets(len(th), 2, 4, seed=5)
    f0 = np.zeros_like(f_gt)
    _, _, o0 = oracle_solver(w, tol=1e-13, f=f0)
    g0 = o0.gradient(th, rec, y)[1]
    gamma = 0.05 / float(np.max(np.abs(g0)))
    tau = 0.004 / gamma
    ref_losses = []

    def grad_fn(fb, idx):
        _, _, ob = oracle_solver(w, tol=1e-13, f=fb)
        loss, g, _ = ob.gradient(th[idx], rec, y[idx])
        ref_losses.append(loss)
        return g

    ref = O.fbs(grad_fn, f0, subsets, gamma, tau, prox_iters=40)
    s = make_solver(w, B=len(th), maxit=3000)
    f, losses, infos = fbs(s, to_t(th, torch), to_t(rec, torch), to_t(y, torch), to_t(f0, torch), subsets,
                           gamma, tau, prox_iters=40)
    assert np.max(ref) > 0.0 and O.tv(ref) > 0.0
    assert losses == pytest.approx(ref_losses, rel=1e-9)
    assert rel(f.cpu().numpy(), ref) < 1e-8
    assert all(i["converged"] for fw, adj in infos for i in fw + adj)
