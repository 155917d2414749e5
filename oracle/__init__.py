"""FP64 CPU oracle of the multigrid-preconditioned Helmholtz solver (test infrastructure).

This package is test infrastructure, not product code.  Only the test-suite, the smoke
check and the bench's CPU-baseline / reference leg may import it.  It is a plain, slow,
numpy/scipy restatement of the paper's discretisation and solver, written for a reader
to check against the paper by eye:

  helmholtz.py   grid, absorbing layer, five-point operator with Sommerfeld closure
                 (Sec. IV-A), shifted-Laplacian operator K_kappa (Sec. IV-B)
  multigrid.py   damped Jacobi (Sec. III, eq. dampedJ), full weighting and bilinear
                 prolongation (Sec. IV-C), coarse re-discretisation, the MG cycle (Alg. 2)
  krylov.py      right-preconditioned flexible GMRES(m) (Saad & Schultz; Saad 1993), the
                 paper's preconditioned Bi-CGSTAB (Alg. 3), its s-step, deflated-restart and
                 IDR(s) relatives
  tomography.py  plane-wave incident field and right-hand side (Sec. II-A), truncation to
                 Omega, receiver sampling, the quadratic data term (Sec. V) and its
                 gradient through one adjoint solve per illumination (Prop. 1)

Everything runs in float64 / complex128.  The oracle shares no code with the CUDA path;
both take their inputs from the `workloads` module.
"""
from .helmholtz import Problem, absorbing_factor, fine_coefficient, operator_diagonal, apply_operator, assemble_operator
from .multigrid import (coarse_size, restrict, prolong, restrict_coefficient, build_hierarchy,
                        jacobi, mg_cycle, Preconditioner)
from .krylov import fgmres, bicgstab, SolveInfo
from .tomography import (incident_field, rhs, crop, embed, sample, misfit, gradient_from_adjoint,
                         MGHSolver, direct_solve)
from .inverse import tv, tv_prox, fbs, snr, grad_fwd, grad_adj

__all__ = [
    "Problem", "absorbing_factor", "fine_coefficient", "operator_diagonal", "apply_operator",
    "assemble_operator", "coarse_size", "restrict", "prolong", "restrict_coefficient",
    "build_hierarchy", "jacobi", "mg_cycle", "Preconditioner", "fgmres", "bicgstab", "SolveInfo",
    "incident_field", "rhs", "crop", "embed", "sample", "misfit", "gradient_from_adjoint",
    "MGHSolver", "direct_solve", "tv", "tv_prox", "fbs", "snr", "grad_fwd", "grad_adj",
]
