"""Parity of the CycleType >= 2 cycles (Alg. 2: W-cycle and CycleType 3) and of per-level sweep
counts with the FP64 oracle, through the C ABI.

Tolerances as for the V-cycle: the FP64 cycle agrees with the oracle's to rounding (relative L2
<= 1e-12); the FP32 cycle within 1e-5; solves preconditioned by a W-cycle reach the direct
solution within 1e-10 (FP64) and 1e-5 (mixed), and the FP64 path takes the oracle's step count.
The grid (70 x 53 interior + 9-cell layer = 88 x 71 points) is ragged against every tile shape.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import make_solver, oracle_solver, rel, torch_cuda

pytestmark = pytest.mark.gpu


def ragged(precision="fp64", levels=4, n_angles=3, **kw):
    return W.Workload("ragged", 70, 53, 9, 8.0, n_angles, -50.0, 40.0, "ellipses", 11, levels=levels,
                      nu1=1, nu2=1, precision=precision, **kw)


def to_t(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    (2, 4, 1, 1),                          # W-cycle, uniform sweeps
    (2, 4, [2, 1, 1], [1, 2, 1]),          # W-cycle, per-level sweeps
    (3, 4, 2, 1),                          # CycleType 3
    (1, 4, [0, 2, 3], [3, 0, 1]),          # V-cycle, per-level sweeps (including 0 on a level)
    (2, 5, [1, 1, 2, 1], [1, 2, 1, 1]),    # deeper W-cycle
    (2, 2, 2, 2),                          # two levels: the two-grid cycle
]


@pytest.mark.parametrize("gamma,levels,nu1,nu2", CASES)
def test_cycle_fp64_matches_oracle(gamma, levels, nu1, nu2):
    torch = torch_cuda()
    w = ragged(levels=levels)
    if levels == 2:
        w = W.Workload("ragged2", 30, 21, 5, 8.0, 3, 0, 0, "ellipses", 12, levels=2, nu1=1, nu2=1,
                       precision="fp64")
    s = make_solver(w, B=4, nu1=nu1, nu2=nu2, cycle_type=gamma)
    pad = lambda nu: nu if isinstance(nu, int) else list(nu) + [0]
    p, f, o = oracle_solver(w, nu1=pad(nu1), nu2=pad(nu2), cycle_type=gamma)
    s.set_contrast(to_t(f, torch))
    b = W.random_field((3, p.ny, p.nx), 13)
    z = s.precondition(to_t(b, torch)).cpu().numpy()
    for q in range(3):
        assert rel(z[q], o.M(b[q])) < 1e-12, (q, rel(z[q], o.M(b[q])))


@pytest.mark.parametrize("gamma,levels,nu1,nu2", [CASES[1], CASES[2], CASES[4]])
def test_cycle_mixed32_matches_oracle(gamma, levels, nu1, nu2):
    torch = torch_cuda()
    w = ragged(levels=levels, precision="mixed32")
    s = make_solver(w, B=3, nu1=nu1, nu2=nu2, cycle_type=gamma)
    pad = lambda nu: nu if isinstance(nu, int) else list(nu) + [0]
    p, f, o = oracle_solver(w, nu1=pad(nu1), nu2=pad(nu2), cycle_type=gamma)
    s.set_contrast(to_t(f, torch))
    b = W.random_field((3, p.ny, p.nx), 14)
    z = s.precondition(to_t(b, torch)).cpu().numpy()
    for q in range(3):
        assert rel(z[q], o.M(b[q])) < 1e-5


@pytest.mark.parametrize("precision,tol,bound,arnoldi", [("fp64", 1e-12, 1e-10, "auto"),
                                                         ("mixed32", 1e-10, 1e-5, "sstep"),
                                                         ("mixed32", 1e-10, 1e-5, "df")])
def test_w_cycle_solve_matches_direct_solve(precision, tol, bound, arnoldi):
    torch = torch_cuda()
    w = ragged(precision=precision, levels=4, restart=8, tol=tol)
    s = make_solver(w, B=4, maxit=3000, cycle_type=2, arnoldi=arnoldi)
    p, f, o = oracle_solver(w)
    s.set_contrast(to_t(f, torch))
    th = W.angles(w)
    b = np.stack([O.rhs(p, f, t) for t in th])
    x, infos = s.solve(to_t(b, torch))
    x = x.cpu().numpy()
    for q in range(len(th)):
        assert infos[q]["converged"] and infos[q]["rel_residual"] <= tol
        assert rel(x[q], O.direct_solve(p, o.D, b[q])) < bound
        true = np.linalg.norm(b[q] - o.apply_A(x[q])) / np.linalg.norm(b[q])
        assert true <= tol * (1 + 1e-6)


def test_w_cycle_fp64_step_count_matches_oracle():
    """FP64 FGMRES(8) with a W-cycle takes the oracle's step count (same arithmetic up to
    rounding), and not more steps than with a V-cycle (up to 2)."""
    torch = torch_cuda()
    w = ragged(levels=4, restart=8, tol=1e-8)
    p, f, o = oracle_solver(w, tol=1e-8, restart=8, cycle_type=2)
    b = O.rhs(p, f, 0.3)
    _, ref = o.solve(b)
    steps = {}
    for gamma in (1, 2):
        s = make_solver(w, B=1, maxit=6000, cycle_type=gamma)
        s.set_contrast(to_t(f, torch))
        _, infos = s.solve(to_t(b[None], torch))
        assert infos[0]["converged"]
        steps[gamma] = infos[0]["iterations"]
    assert ref.converged and abs(steps[2] - ref.iterations) <= 1, (steps, ref.iterations)
    assert steps[2] <= steps[1] + 2


@pytest.mark.parametrize("precision,gamma,bound", [("fp64", 1, 1e-13), ("fp64", 2, 1e-13), ("mixed32", 1, 1e-5),
                                                   ("mixed32", 3, 1e-5)])
def test_one_kernel_coarse_tail_matches_level_kernels(precision, gamma, bound, monkeypatch):
    """The coarse tail in one kernel (every level from the first that fits in shared memory) gives
    the cycle of the level-by-level kernels (MGH_TAIL=0): same FP64 arithmetic to rounding, FP32
    within the FP32 cycle's bound; on this grid the tail starts at level 1."""
    torch = torch_cuda()
    w = ragged(levels=4, precision=precision)
    p, f, o = oracle_solver(w, nu1=[2, 1, 1, 0], nu2=[1, 2, 1, 0], cycle_type=gamma)
    b = W.random_field((3, p.ny, p.nx), 15)
    z = {}
    for tail in ("1", "0"):
        monkeypatch.setenv("MGH_TAIL", tail)
        s = make_solver(w, B=3, nu1=[2, 1, 1], nu2=[1, 2, 1], cycle_type=gamma)
        s.set_contrast(to_t(f, torch))
        z[tail] = s.precondition(to_t(b, torch)).cpu().numpy()
        s.close()
    for q in range(3):
        assert rel(z["1"][q], z["0"][q]) < bound
        assert rel(z["1"][q], o.M(b[q])) < (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed32"])
@pytest.mark.parametrize("levels,gamma", [(4, 1), (4, 2), (5, 1)])
def test_cluster_tail_equals_the_one_block_tail_bit_for_bit(precision, levels, gamma):
    """The coarse tail split over a cluster of 2 or 4 blocks per right-hand side (bands of rows, halo
    rows through distributed shared memory, each block forming its rows of the coarsest product)
    computes every point with the one-block tail's operations.  On this grid the fourth block of a
    4-block cluster owns no row of the tail's finest level, and with 4 levels none of the lower
    levels either."""
    torch = torch_cuda()
    w = ragged(levels=levels, precision=precision)
    p = O.Problem.from_workload(w)
    f = W.phantom(w)
    b = W.random_field((3, p.ny, p.nx), 16)
    s = make_solver(w, B=3, cycle_type=gamma)
    s.set_contrast(to_t(f, torch))
    base = s.kernel_shape()
    assert base["tail_level"] >= 1 and base["tail_cluster"] == 0   # automatic
    s.set_kernel_shape(**dict(base, tail_cluster=1))
    z1 = s.precondition(to_t(b, torch)).cpu().numpy()
    for cl in (2, 4, 0):
        s.set_kernel_shape(**dict(base, tail_cluster=cl))
        assert s.kernel_shape()["tail_cluster"] == cl
        np.testing.assert_array_equal(s.precondition(to_t(b, torch)).cpu().numpy(), z1)
    s.close()
