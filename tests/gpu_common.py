"""Shared helpers of the GPU parity tests (inputs from workloads, references from oracle)."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_solver(w, B=None, **kw):
    torch = torch_cuda()
    from paper_2107_03679_gb300 import Solver
    return Solver.from_workload(w, batch_max=B or w.n_angles, device=torch.device("cuda", 0), **kw)


def oracle_solver(w, tol=1e-12, f=None, **kw):
    p = O.Problem.from_workload(w)
    f = W.phantom(w) if f is None else f
    args = dict(levels=w.levels, nu1=w.nu1, nu2=w.nu2, omega=w.omega,
                shift=complex(w.shift_re, w.shift_im), restart=w.restart, tol=tol)
    args.update(kw)
    return p, f, O.MGHSolver(p, f, **args)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))
