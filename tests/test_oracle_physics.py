"""Physics pin of the oracle's discretisation against the paper's worked example (Sec. VI-A):
a dielectric disk (eta = 2.2, radius 1.25 wavelengths) in air, 256^2 points over 3.2 wavelengths,
a 32-point absorbing layer with beta = 0.15.  The paper reports a squared relative error of
7.5e-3 for the total field of its Helmholtz model against the analytic solution.  The oracle's
discrete solution (same discretisation, exact sparse solve) is compared with the analytic
series of a dielectric cylinder under plane-wave illumination (TM, e^{-j w t})."""
import json
import math
import os

import numpy as np
import scipy.special as ssp

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_disk_e1.json")


def cylinder_total_field(k0, eta, R, x, y, nmax):
    """Total field of a plane wave e^{j k0 x} scattered by a dielectric cylinder of radius R centred
    at the origin: outside sum_n j^n [J_n(k0 r) + a_n H_n(k0 r)] e^{j n phi}, inside
    sum_n j^n c_n J_n(k1 r) e^{j n phi}, coefficients from continuity of u and du/dr at r = R."""
    k1 = k0 * eta
    r = np.hypot(x, y)
    phi = np.arctan2(y, x)
    u = np.zeros(r.shape, dtype=np.complex128)
    inside = r <= R
    for n in range(-nmax, nmax + 1):
        J0, J0p = ssp.jv(n, k0 * R), ssp.jvp(n, k0 * R)
        J1, J1p = ssp.jv(n, k1 * R), ssp.jvp(n, k1 * R)
        H0, H0p = ssp.hankel1(n, k0 * R), ssp.h1vp(n, k0 * R)
        a = (k1 * J1p * J0 - k0 * J1 * J0p) / (k0 * J1 * H0p - k1 * J1p * H0)
        c = (J0 + a * H0) / J1
        ph = (1j ** n) * np.exp(1j * n * phi)
        u[~inside] += ph[~inside] * (ssp.jv(n, k0 * r[~inside]) + a * ssp.hankel1(n, k0 * r[~inside]))
        u[inside] += ph[inside] * c * ssp.jv(n, k1 * r[inside])
    return u


def test_series_reduces_to_plane_wave_without_contrast():
    k0 = 2 * math.pi / 80.0
    x, y = np.meshgrid(np.arange(-50, 50, 7.0), np.arange(-40, 60, 9.0))
    u = cylinder_total_field(k0, 1.0, 30.0, x, y, 60)
    np.testing.assert_allclose(u, np.exp(1j * k0 * x), atol=1e-10)


def test_disk_total_field_matches_paper_error_level():
    g = json.load(open(GOLDEN))
    n_int = g["grid_points_per_side"]
    ppw = g["wavelength_cm"] / g["h_cm"]                      # 80 points per wavelength
    k = 2 * math.pi / ppw
    R = g["radius_wavelengths"] * ppw                          # 100 cells
    p = O.Problem(n_int, n_int, g["abl_points_per_side"], h=1.0, k=k, beta=g["beta"])
    c0 = (n_int - 1) / 2.0
    m = np.arange(n_int)[None, :] - c0
    n = np.arange(n_int)[:, None] - c0
    f_d = np.where(m ** 2 + n ** 2 <= R ** 2, g["eta_disk"] ** 2 - 1.0, 0.0)
    c = O.fine_coefficient(p, f_d)
    D = O.operator_diagonal(c, O.absorbing_factor(p), p.h, p.k)
    u_sc = O.direct_solve(p, D, O.rhs(p, f_d, 0.0))
    u_tot = O.crop(p, u_sc + O.incident_field(p, 0.0))
    # analytic field at the same grid points, phase referred to grid index 0 of Omega_e
    x = m + c0 + p.abl
    ref = cylinder_total_field(k, g["eta_disk"], R, np.broadcast_to(m, (n_int, n_int)),
                               np.broadcast_to(n, (n_int, n_int)), 80)
    ref = ref * np.exp(1j * k * (c0 + p.abl))                  # incident phase e^{j k x}, x from index 0
    eps = float(np.sum(np.abs(u_tot - ref) ** 2) / np.sum(np.abs(ref) ** 2))
    # same discretisation as the paper: the error lands within +-50 % of the paper's 7.5e-3
    # (the oracle gives 9.2e-3); a wrong damping sign or a misplaced closure is far outside
    assert 0.5 * g["relative_error_MGH"] < eps < 1.5 * g["relative_error_MGH"], eps
