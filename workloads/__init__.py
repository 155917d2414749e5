"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only draws inputs: grid geometry, contrast phantoms f_d = (n/n_b)^2 - 1,
illumination angles and receiver index sets.  It holds none of the method's arithmetic
(no operator, no right-hand side, no solve), so both sides of every parity test can
take their inputs from here without sharing any solver code.

The workloads stand in for the paper's experiments (Sec. VI): plane-wave illumination
of a dielectric object in a homogeneous background, discretised on a uniform grid with
an absorbing boundary layer around the region of interest (Sec. IV-A).  The paper's own
phantom image, its sweep data and the Fresnel measurements are not used; every input is
drawn from a fixed seed with numpy's default generator.

Conventions (shared by both sides):
  * fields are stored row-major [ny][nx] with x (index m) fastest, idx = n*nx + m;
  * the contrast f_d lives on the interior region Omega, shape [ny_int][nx_int];
  * lengths are in grid cells (h = 1) unless a workload says otherwise, so the
    background wavenumber is k = 2*pi/ppw for ppw points per wavelength.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict, replace
from typing import List, Optional

import numpy as np


@dataclass
class Workload:
    """Geometry, solver settings and inputs of one synthetic configuration."""
    name: str
    nx_int: int
    ny_int: int
    abl: int
    ppw: float                 # background points per wavelength (k*h = 2*pi/ppw)
    n_angles: int
    angle_lo_deg: float
    angle_hi_deg: float
    phantom: str               # generator name, see phantom()
    seed: int
    levels: int
    nu1: int
    nu2: int
    omega: float = 0.8
    shift_re: float = 1.0
    shift_im: float = 0.5
    beta: float = 0.15
    restart: int = 20
    tol: float = 1e-6
    precision: str = "mixed32"  # "fp64" | "mixed32" | "mixed16"
    h: float = 1.0
    krylov: str = "fgmres"      # outer method: "fgmres" | "bicgstab" (Alg. 3) | "idrs"
    extra: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return self.nx_int + 2 * self.abl

    @property
    def ny(self) -> int:
        return self.ny_int + 2 * self.abl

    @property
    def k(self) -> float:
        return 2.0 * math.pi / (self.ppw * self.h)

    def to_dict(self) -> dict:
        d = asdict(self)
        d["nx"], d["ny"], d["k"] = self.nx, self.ny, self.k
        return d


# The five configurations of the hot path, with their synthetic inputs.
WORKLOADS = {
    # Plain method, single solve: 128^2 + 16-cell layer, centred disk r=20, n/nb=1.05,
    # one plane wave along +x, FP64, GMRES(20), shift 1+0.5i, 4 levels, 2+2 sweeps.
    "disk160": Workload("disk160", 128, 128, 16, 10.0, 1, 0.0, 0.0, "disk", 1,
                        levels=4, nu1=2, nu2=2, restart=20, tol=1e-8, precision="fp64"),
    # Batched forward, mixed precision: 512^2 + 32, sum of 6 random ellipses, 60 angles.
    # GMRES restart 8: on this workload the oracle needs 649 / 655 / 666 / 667 / 692 steps for
    # m = 20 / 16 / 10 / 8 / 5 (nu = 1), while the cost of a step grows with m.  Two smoothing
    # sweeps: 603 steps per solve on the GPU against 675 with one and 625 with three.
    "ellipses576": Workload("ellipses576", 512, 512, 32, 10.0, 60, -60.0, 60.0,
                            "ellipses", 2, levels=6, nu1=2, nu2=2, restart=8, tol=1e-6),
    # Strong scattering: 1024^2 + 48, cell-like phantom, 120 angles, 12 ppw.  Restarted FGMRES
    # stagnates at this contrast; the paper's Bi-CGSTAB (Alg. 3) with kappa = 1 + 1j converges with
    # the FP64 cycle (with the FP32 cycle its short recurrences do not), so the FP64 path is the
    # workload's setting.  A forward problem: its bench step is set_contrast + forward solves.
    "cell1120": Workload("cell1120", 1024, 1024, 48, 12.0, 120, -70.0, 70.0,
                         "cell", 3, levels=7, nu1=2, nu2=2, restart=8, tol=1e-6, shift_im=1.0,
                         krylov="bicgstab", precision="fp64", extra={"forward_only": True}),
    # Differentiation: 512^2 + 32, ground-truth ellipse, 60 angles, receivers on a line.
    "grad576": Workload("grad576", 512, 512, 32, 10.0, 60, -60.0, 60.0,
                        "gt_ellipse", 4, levels=6, nu1=2, nu2=2, restart=8, tol=1e-6),
}


def uneven_workloads() -> List[Workload]:
    """Uneven batch: four grids solved together, each with its own angles (absorbing layer of
    n/16 cells per side, 10 points per wavelength, seeded ellipse phantoms with n/n_b <= 1.2).
    Levels are chosen so that the coarsest grid has 18-36 points per side."""
    spec = [(256, 90, 5, 51), (384, 60, 5, 52), (768, 40, 6, 53), (2048, 16, 8, 54)]
    return [Workload(f"uneven{n}", n, n, n // 16, 10.0, b, -60.0, 60.0, "ellipses", seed, levels=lv,
                     nu1=2, nu2=2, restart=8, tol=1e-6) for n, b, lv, seed in spec]


def multifrequency_workloads(w: Workload, freqs=(3.0, 5.0, 6.0, 8.0)) -> List[Workload]:
    """One contrast illuminated at several frequencies on w's grid (Sec. VI-C uses 3, 5, 6 and 8
    GHz): the highest frequency has w's points per wavelength, a lower frequency f proportionally
    more (ppw * f_max / f); everything else, the phantom and its seed included, is w's."""
    fmax = max(freqs)
    return [replace(w, name=f"{w.name}@{f:g}", ppw=w.ppw * fmax / f) for f in freqs]


def small_workload(name: str = "small", n_int: int = 40, abl: int = 6, ppw: float = 10.0,
                   n_angles: int = 3, levels: int = 3, phantom: str = "ellipses",
                   seed: int = 7, precision: str = "fp64", **kw) -> Workload:
    """A reduced configuration of the same structure, sized for the oracle to finish in seconds."""
    w = Workload(name, n_int, n_int, abl, ppw, n_angles, -60.0, 60.0, phantom, seed,
                 levels=levels, nu1=kw.pop("nu1", 1), nu2=kw.pop("nu2", 1),
                 precision=precision, **kw)
    return w


def angles(w: Workload) -> np.ndarray:
    """Illumination angles theta (radians, from +x, counter-clockwise), evenly spaced."""
    if w.n_angles == 1:
        return np.array([math.radians(w.angle_lo_deg)], dtype=np.float64)
    return np.radians(np.linspace(w.angle_lo_deg, w.angle_hi_deg, w.n_angles)).astype(np.float64)


def _ellipse_mask(nx: int, ny: int, cx: float, cy: float, a: float, b: float, rot: float) -> np.ndarray:
    """Grid points (m, n) of the interior lying inside the rotated ellipse (membership at grid points)."""
    m = np.arange(nx, dtype=np.float64)[None, :]
    n = np.arange(ny, dtype=np.float64)[:, None]
    dx, dy = m - cx, n - cy
    c, s = math.cos(rot), math.sin(rot)
    u = c * dx + s * dy
    v = -s * dx + c * dy
    return (u / a) ** 2 + (v / b) ** 2 <= 1.0


def _scale_lengths(n_int: int, ref: int, lo: float, hi: float):
    s = n_int / ref
    return lo * s, hi * s


def phantom(w: Workload) -> np.ndarray:
    """Contrast f_d = (n/n_b)^2 - 1 on the interior, float64 [ny_int][nx_int], drawn from w.seed.

    Generators (lengths scale with the interior size relative to the named workload):
      disk        centred disk of radius 20 cells (x n_int/128), n/n_b = 1.05.
      ellipses    6 ellipses, n/n_b ~ U[1.0, 1.2], semi-axes ~ U[20, 120] cells (x n_int/512),
                  rotation ~ U[0, pi), centre uniform such that the ellipse stays inside;
                  overlapping contributions add.
      cell        outer ellipse n/n_b = 1.3 (semi-axes ~ U[0.35, 0.45] n_int), and 10 disks
                  inside it, radius ~ U[0.02, 0.06] n_int, n/n_b ~ U[1.3, 1.5], replacing it.
      gt_ellipse  one ellipse, semi-axes ~ U[0.12, 0.25] n_int, n/n_b ~ U[1.05, 1.15],
                  centred within the left 60 % of the interior.
    """
    rng = np.random.default_rng(w.seed)
    nx, ny = w.nx_int, w.ny_int
    f = np.zeros((ny, nx), dtype=np.float64)
    if w.phantom == "disk":
        r = 20.0 * nx / 128.0
        mask = _ellipse_mask(nx, ny, (nx - 1) / 2.0, (ny - 1) / 2.0, r, r, 0.0)
        f[mask] = 1.05 ** 2 - 1.0
    elif w.phantom == "ellipses":
        lo, hi = _scale_lengths(min(nx, ny), 512, 20.0, 120.0)
        for _ in range(6):
            ratio = rng.uniform(1.0, 1.2)
            a, b = rng.uniform(lo, hi), rng.uniform(lo, hi)
            rot = rng.uniform(0.0, math.pi)
            R = max(a, b)
            cx = rng.uniform(R, nx - 1 - R)
            cy = rng.uniform(R, ny - 1 - R)
            f[_ellipse_mask(nx, ny, cx, cy, a, b, rot)] += ratio ** 2 - 1.0
    elif w.phantom == "cell":
        n = min(nx, ny)
        a, b = rng.uniform(0.35 * n, 0.45 * n), rng.uniform(0.35 * n, 0.45 * n)
        rot = rng.uniform(0.0, math.pi)
        cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
        outer = _ellipse_mask(nx, ny, cx, cy, a, b, rot)
        f[outer] = 1.3 ** 2 - 1.0
        rmin = min(a, b)
        for _ in range(10):
            r = rng.uniform(0.02 * n, 0.06 * n)
            rho = rng.uniform(0.0, max(rmin - r, 0.0))
            phi = rng.uniform(0.0, 2.0 * math.pi)
            ratio = rng.uniform(1.3, 1.5)
            disk = _ellipse_mask(nx, ny, cx + rho * math.cos(phi), cy + rho * math.sin(phi), r, r, 0.0)
            f[disk] = ratio ** 2 - 1.0
    elif w.phantom == "gt_ellipse":
        n = min(nx, ny)
        a, b = rng.uniform(0.12 * n, 0.25 * n), rng.uniform(0.12 * n, 0.25 * n)
        rot = rng.uniform(0.0, math.pi)
        ratio = rng.uniform(1.05, 1.15)
        R = max(a, b)
        cx = rng.uniform(R, max(R, 0.6 * nx - R))
        cy = rng.uniform(R, ny - 1 - R)
        f[_ellipse_mask(nx, ny, cx, cy, a, b, rot)] = ratio ** 2 - 1.0
    elif w.phantom == "zero":
        pass
    elif w.phantom == "random":
        f[:] = rng.uniform(0.0, 0.3, size=(ny, nx))
    else:
        raise ValueError(f"unknown phantom {w.phantom!r}")
    return f


def receivers(w: Workload, f_gt: Optional[np.ndarray] = None) -> np.ndarray:
    """Receiver grid indices (int64, flat index n*nx + m on the extended grid).

    One vertical line shared by all angles, 10 cells beyond the far (+x) side of the
    ground-truth object's bounding box, covering every interior row.  All illumination
    angles lie within +-70 degrees of +x, so this line sees the forward-scattered field.
    """
    if f_gt is None:
        f_gt = phantom(w)
    cols = np.nonzero(np.any(f_gt != 0.0, axis=0))[0]
    xmax = int(cols.max()) if cols.size else w.nx_int // 2
    m_int = min(xmax + 10, w.nx_int - 1)
    m = w.abl + m_int
    n = w.abl + np.arange(w.ny_int, dtype=np.int64)
    return (n * w.nx + m).astype(np.int64)


def complex_noise(shape, sigma: float, seed: int) -> np.ndarray:
    """Circular complex Gaussian noise sigma*(xi1 + j*xi2)/sqrt(2) from a fixed seed."""
    rng = np.random.default_rng(seed)
    return sigma * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def random_field(shape, seed: int) -> np.ndarray:
    """A seeded complex128 test field with independent N(0,1) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def angle_subsets(n_angles: int, subset: int, iters: int, seed: int = 0):
    """The angle indices of each reconstruction iteration: `subset` of the n_angles drawn without
    replacement (sorted) from default_rng(seed), one draw per iteration; all angles when subset is
    0 or at least n_angles."""
    if subset <= 0 or subset >= n_angles:
        return [np.arange(n_angles) for _ in range(iters)]
    rng = np.random.default_rng(seed)
    return [np.sort(rng.choice(n_angles, subset, replace=False)) for _ in range(iters)]


def fmix32(h: np.ndarray) -> np.ndarray:
    """MurmurHash3's 32-bit finaliser (Appleby): h ^= h >> 16; h *= 0x85EBCA6B; h ^= h >> 13;
    h *= 0xC2B2AE35; h ^= h >> 16, all modulo 2^32."""
    h = np.asarray(h).astype(np.uint32)
    h = h ^ (h >> np.uint32(16))
    h = h * np.uint32(0x85EBCA6B)
    h = h ^ (h >> np.uint32(13))
    h = h * np.uint32(0xC2B2AE35)
    return h ^ (h >> np.uint32(16))


def idr_shadow(n_points: int, s: int) -> np.ndarray:
    """The shadow space of IDR(s) (random numbers the method draws), n_points x s: entry (q, i) is
    (1 - 2 b_{2i}) + j (1 - 2 b_{2i+1}) with b the bits of fmix32(q + 0x9E3779B9 mod 2^32), q the
    point index idx = n*nx + m.  The CUDA engine generates the same entries from the same
    published finaliser; a test hands this matrix to the oracle as its shadow space."""
    if not 1 <= s <= 16:
        raise ValueError("idr_shadow: 1 <= s <= 16")
    q = np.arange(n_points, dtype=np.uint64)
    bits = fmix32(((q + np.uint64(0x9E3779B9)) & np.uint64(0xFFFFFFFF)).astype(np.uint32))
    P = np.empty((n_points, s), dtype=np.complex128)
    for i in range(s):
        a = (bits >> np.uint32(2 * i)) & np.uint32(1)
        b = (bits >> np.uint32(2 * i + 1)) & np.uint32(1)
        P[:, i] = (1.0 - 2.0 * a) + 1j * (1.0 - 2.0 * b)
    return P
