"""Per-level smoothing sweep counts from the local Fourier analysis of damped Jacobi on K_kappa.

On level l (spacing 2^l h) of the background medium, with q = (k 2^l h)^2, one damped-Jacobi sweep
multiplies the Fourier mode whose Laplacian symbol is lam = 4 - 2 cos t1 - 2 cos t2 (in [0, 8]) by

    s(lam) = 1 - omega (lam - kappa q) / (4 - kappa q)

(the smoothing analysis of Sec. IV-B with the shift kappa).  s is affine in lam, so its largest
modulus is reached at lam = 0 or lam = 8.  For the Helmholtz operator it exceeds 1 (the smoother
amplifies some mode); the amplification grows as q approaches 4, where the diagonal 4 - kappa q is
smallest.  A level with amplification a > 1 per sweep gets at most floor(log A / log a) sweeps
(and at least one), A being the growth tolerated in one smoothing phase; the remark after Alg. 2
allows the counts to differ by level.  With A = 2.5 a grid with 10 points per wavelength keeps two
sweeps on every level (largest a = 1.45, level 1), while a level at q = 3.55 (a = 1.81) gets one:
with two sweeps there, FGMRES(8) on the 576^2 ellipse contrast at 13.3 points per wavelength stalls
(relative residual 0.63 after 1,500 steps), with one it converges in 390.

Host-side parameter choice only: the solver's arithmetic is in the CUDA library.
"""
from __future__ import annotations

import math
from typing import List


def jacobi_amplification(q: float, omega: float = 0.8, shift: complex = 1.0 + 0.5j) -> float:
    """max over Fourier modes of |s| for (k h)^2 = q on a level of the background medium."""
    d = 4.0 - shift * q
    return max(abs(1.0 - omega * (lam - shift * q) / d) for lam in (0.0, 8.0))


def smoothing_sweeps(k: float, h: float, levels: int, nu: int, omega: float = 0.8, shift: complex = 1.0 + 0.5j,
                     growth: float = 2.5) -> List[int]:
    """Sweeps for levels 0 .. levels-2 (the coarsest is solved exactly): nu, capped on the levels
    whose smoother amplifies by more than `growth` in nu sweeps."""
    out = []
    for l in range(levels - 1):
        a = jacobi_amplification((k * h * 2 ** l) ** 2, omega, shift)
        n = nu if a <= 1.0 else min(nu, max(1, int(math.log(growth) / math.log(a))))
        out.append(n)
    return out
