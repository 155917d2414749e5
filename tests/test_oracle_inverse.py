"""Pins of the reconstruction oracle (Sec. V, Alg. 4): the TV proximal operator by fast gradient
projection against closed forms and optimality, the accelerated FBS recursion by hand, SNR."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def test_difference_operators_are_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((7, 9))
    p, q = rng.standard_normal((7, 9)), rng.standard_normal((7, 9))
    gp, gq = O.grad_fwd(x)
    assert abs(np.vdot(gp, p) + np.vdot(gq, q) - np.vdot(x, O.grad_adj(p, q))) < 1e-12


def test_prox_without_tv_is_the_clamp():
    w = np.array([[0.5, -0.2], [1.0, -3.0]])
    np.testing.assert_array_equal(O.tv_prox(w, 0.0, 10), np.maximum(w, 0.0))


@pytest.mark.parametrize("b1,b2,lam", [(1.0, 0.2, 0.1), (1.0, 0.2, 0.5), (0.3, 0.25, 0.2)])
def test_prox_two_pixels_closed_form(b1, b2, lam):
    """One difference: min 1/2 ||x - b||^2 + lam |x1 - x2| moves each value by lam toward the other,
    or merges them at the mean when they are closer than 2 lam."""
    x = O.tv_prox(np.array([[b1, b2]]), lam, 3000)[0]
    if b1 - b2 > 2 * lam:
        ref = [b1 - lam, b2 + lam]
    else:
        ref = [(b1 + b2) / 2] * 2
    np.testing.assert_allclose(x, ref, atol=1e-6)


def test_prox_step_closed_form():
    """A 1 x 8 step (a on 4 pixels, b on 4) keeps its jump and each side moves by lam / 4."""
    a, b, lam = 1.0, 0.1, 0.4
    w = np.array([[a] * 4 + [b] * 4])
    x = O.tv_prox(w, lam, 3000)[0]
    np.testing.assert_allclose(x, [a - lam / 4] * 4 + [b + lam / 4] * 4, atol=1e-6)


def test_prox_is_optimal_on_a_random_image():
    """The objective at the prox output is not lowered by any small feasible perturbation."""
    rng = np.random.default_rng(2)
    w = rng.standard_normal((12, 10)) * 0.5 + 0.3
    lam = 0.2
    x = O.tv_prox(w, lam, 4000)
    obj = lambda z: 0.5 * np.sum((z - w) ** 2) + lam * O.tv(z)
    f0 = obj(x)
    assert np.all(x >= 0)
    for _ in range(60):
        z = np.maximum(x + 1e-3 * rng.standard_normal(x.shape), 0.0)
        assert obj(z) >= f0 - 1e-7
    assert f0 < obj(np.maximum(w, 0.0))


def test_fbs_recursion_by_hand():
    """Alg. 4 on the separable toy 1/2 ||f - c||^2 with tau = 0 (prox = clamp): the first iterates
    and the momentum coefficients written out."""
    c = np.array([[0.7, -0.3, 0.2]])
    grad = lambda f, idx: f - c
    gamma = 0.4
    seen = []
    O.fbs(grad, np.zeros_like(c), [np.arange(1)] * 3, gamma, 0.0, callback=lambda it, f: seen.append(f.copy()))
    f1 = np.maximum(0 - gamma * (0 - c), 0)
    a2 = (1 + np.sqrt(5)) / 2
    fb2 = f1 + (1 - 1) / a2 * (f1 - 0)
    f2 = np.maximum(fb2 - gamma * (fb2 - c), 0)
    a3 = (1 + np.sqrt(1 + 4 * a2 * a2)) / 2
    fb3 = f2 + (a2 - 1) / a3 * (f2 - f1)
    f3 = np.maximum(fb3 - gamma * (fb3 - c), 0)
    np.testing.assert_allclose(seen[0], f1, atol=1e-15)
    np.testing.assert_allclose(seen[1], f2, atol=1e-15)
    np.testing.assert_allclose(seen[2], f3, atol=1e-15)


def test_snr_definition():
    x = np.array([3.0, 4.0])
    assert O.snr(1.1 * x, x) == pytest.approx(20.0)
    assert O.snr(np.zeros(2), x) == pytest.approx(0.0)


def test_angle_subsets():
    s = W.angle_subsets(60, 8, 5, seed=3)
    assert len(s) == 5 and all(len(a) == 8 and len(set(a)) == 8 and a.max() < 60 for a in s)
    assert all(np.array_equal(a, b) for a, b in zip(s, W.angle_subsets(60, 8, 5, seed=3)))
    assert all(len(a) == 60 for a in W.angle_subsets(60, 0, 2))
