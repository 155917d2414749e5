"""Per-level sweep counts from the LFA of damped Jacobi on K_kappa (CPU only).

The amplification is pinned to the oracle's own Jacobi sweep applied to Fourier modes on a
constant background, and the rule's purpose to the oracle's FGMRES: on a 128^2 + 16 grid at 13.3
points per wavelength (level 2 at (k h_2)^2 = 3.55), two sweeps on every level stall while the
rule's counts converge.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2107_03679_gb300.sweeps import jacobi_amplification, smoothing_sweeps


@pytest.mark.parametrize("ppw,shift", [(10.0, 1 + 0.5j), (5.0, 1 + 0.5j), (3.54, 1 + 0.5j), (2.5, 1 + 0.5j),
                                       (10.0, 1.0 + 0.0j)])
def test_amplification_is_the_largest_jacobi_factor_of_the_oracle(ppw, shift):
    p = O.Problem(24, 24, 4, h=1.0, k=2 * math.pi / ppw)
    c = O.fine_coefficient(p, np.zeros((p.ny_int, p.nx_int)))
    lv = O.build_hierarchy(p, c, 1, shift)[0]
    mask = np.zeros((p.ny, p.nx), dtype=bool)
    mask[p.abl:p.ny - p.abl, p.abl:p.nx - p.abl] = True
    m, n = np.arange(p.nx)[None, :], np.arange(p.ny)[:, None]
    best = 0.0
    for t1 in np.linspace(-math.pi, math.pi, 17):
        for t2 in np.linspace(-math.pi, math.pi, 17):
            e = np.exp(1j * (t1 * m + t2 * n))
            e1 = O.jacobi(lv, np.zeros_like(e), e, 0.8)
            best = max(best, float(np.max(np.abs(e1[mask] / e[mask]))))
    assert jacobi_amplification((p.k * p.h) ** 2, 0.8, shift) == pytest.approx(best, rel=1e-12)


def test_rule_keeps_ten_points_per_wavelength_and_caps_the_amplifying_level():
    k = lambda ppw: 2 * math.pi / ppw
    assert smoothing_sweeps(k(10.0), 1.0, 6, 2) == [2, 2, 2, 2, 2]
    assert smoothing_sweeps(k(40.0 / 3.0), 1.0, 6, 2) == [2, 2, 1, 2, 2]
    assert smoothing_sweeps(k(80.0 / 3.0), 1.0, 6, 2) == [2, 2, 2, 1, 2]
    assert smoothing_sweeps(k(10.0), 1.0, 6, 1) == [1, 1, 1, 1, 1]


def test_capped_sweeps_converge_where_two_sweeps_stall():
    w = W.Workload("s", 128, 128, 16, 40.0 / 3.0, 1, 0, 0, "ellipses", 2, levels=4, nu1=2, nu2=2, restart=8,
                   tol=1e-6)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    b = O.rhs(p, f, 0.0)
    nu = smoothing_sweeps(p.k, p.h, 4, 2)
    assert nu == [2, 2, 1]
    _, stalled = O.MGHSolver(p, f, 4, 2, 2, 0.8, 1 + 0.5j, 8, 1e-6, maxit=300).solve(b)
    _, capped = O.MGHSolver(p, f, 4, nu + [0], nu + [0], 0.8, 1 + 0.5j, 8, 1e-6, maxit=300).solve(b)
    assert not stalled.converged and stalled.rel_residual > 0.1
    assert capped.converged and capped.iterations <= 200
