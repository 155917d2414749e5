"""Direct pins of the oracle's small helpers, each against a brute-force loop written from its
definition (CPU).  They are also exercised through the operator, the multigrid hierarchy and the
solvers; here each one is checked on its own:

* layer_distance_sq: squared Euclidean distance, in fine cells, from a level point's fine position
  to Omega's index box (the absorbing-layer profile beta (d/L)^2 of Sec. IV-A), against the
  minimum over every box point;
* missing_neighbours and neighbour_sum: the five-point stencil's out-of-grid count and in-grid sum
  (Sec. IV-A, the ghost closure and the Laplacian part of a row);
* givens: the rotation of the least-squares updates is unitary and annihilates the second entry;
* restrict_coefficient: full weighting with weights 1/16 [1 2 1; 2 4 2; 1 2 1], samples outside the
  grid as 0, then the outermost coarse ring set to k^2 (Sec. IV-C);
* gradient_from_adjoint: g = k^2 sum_q Re(z_q u_q) on Omega (Prop. 1 with dA = -k^2 diag(df_d)).
"""
import numpy as np
import pytest

import oracle as O
from oracle.helmholtz import layer_distance_sq, missing_neighbours, neighbour_sum
from oracle.krylov import givens
from oracle.multigrid import coarse_size, restrict_coefficient
from oracle.tomography import gradient_from_adjoint


def _problem():
    return O.Problem(5, 4, 3, h=1.0, k=0.7, beta=0.15)   # 11 x 10 extended grid


@pytest.mark.parametrize("scale", [1, 2])
def test_layer_distance_is_the_distance_to_the_box(scale):
    p = _problem()
    nx, ny = (p.nx, p.ny) if scale == 1 else (coarse_size(p.nx), coarse_size(p.ny))
    d2 = layer_distance_sq(p, nx, ny, scale)
    box = [(x, y) for x in range(p.abl, p.abl + p.nx_int) for y in range(p.abl, p.abl + p.ny_int)]
    for j in range(ny):
        for i in range(nx):
            fx, fy = scale * i, scale * j
            best = min((fx - x) ** 2 + (fy - y) ** 2 for x, y in box)
            assert d2[j, i] == best, (i, j)


def test_missing_neighbours_and_neighbour_sum_by_loops():
    ny, nx = 5, 7
    u = np.random.default_rng(3).standard_normal((ny, nx)) + 1j * np.random.default_rng(4).standard_normal((ny, nx))
    cnt = missing_neighbours(nx, ny)
    s = neighbour_sum(u)
    for j in range(ny):
        for i in range(nx):
            miss, acc = 0, 0.0
            for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
                jj, ii = j + dj, i + di
                if 0 <= jj < ny and 0 <= ii < nx:
                    acc += u[jj, ii]
                else:
                    miss += 1
            assert cnt[j, i] == miss
            assert s[j, i] == pytest.approx(acc, abs=1e-14)


@pytest.mark.parametrize("a,b", [(1.0 + 2.0j, -0.5 + 0.25j), (3.0, 4.0), (0.0, 1.0 - 1.0j), (2.0 - 1.0j, 0.0),
                                 (1e-8 + 0j, 5.0 + 3.0j)])
def test_givens_is_unitary_and_annihilates(a, b):
    c, s = givens(complex(a), complex(b))
    G = np.array([[c, s], [-np.conj(s), c]])
    assert np.allclose(G @ G.conj().T, np.eye(2), atol=1e-14)
    out = G @ np.array([a, b], dtype=complex)
    assert abs(out[1]) <= 1e-14 * max(1.0, abs(a) + abs(b))
    assert abs(abs(out[0]) - np.hypot(abs(a), abs(b))) <= 1e-13 * max(1.0, abs(a) + abs(b))


def test_restrict_coefficient_by_its_stencil():
    rng = np.random.default_rng(5)
    for ny, nx in ((9, 11), (8, 10), (7, 6)):
        c = 1.0 + rng.random((ny, nx))
        k = 0.9
        cc = restrict_coefficient(c, k)
        nyc, nxc = coarse_size(ny), coarse_size(nx)
        assert cc.shape == (nyc, nxc)
        w = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]]) / 16.0
        for j in range(nyc):
            for i in range(nxc):
                if j in (0, nyc - 1) or i in (0, nxc - 1):
                    assert cc[j, i] == k ** 2
                    continue
                acc = 0.0
                for dj in (-1, 0, 1):
                    for di in (-1, 0, 1):
                        y, x = 2 * j + dj, 2 * i + di
                        if 0 <= y < ny and 0 <= x < nx:
                            acc += w[dj + 1, di + 1] * c[y, x]
                assert cc[j, i] == pytest.approx(acc, rel=1e-15)


def test_gradient_from_adjoint_by_loops():
    p = _problem()
    rng = np.random.default_rng(6)
    B = 3
    z = rng.standard_normal((B, p.ny, p.nx)) + 1j * rng.standard_normal((B, p.ny, p.nx))
    u = rng.standard_normal((B, p.ny, p.nx)) + 1j * rng.standard_normal((B, p.ny, p.nx))
    g = gradient_from_adjoint(p, z, u)
    assert g.shape == (p.ny_int, p.nx_int)
    for j in range(p.ny_int):
        for i in range(p.nx_int):
            acc = 0.0
            for q in range(B):
                acc += (z[q, p.abl + j, p.abl + i] * u[q, p.abl + j, p.abl + i]).real
            assert g[j, i] == pytest.approx(p.k ** 2 * acc, rel=1e-13)
