"""GB300 (sm_103a) multigrid-preconditioned Helmholtz solver for diffraction tomography.

The solver runs in the CUDA library libmgh.so behind the C ABI of include/mgh.h; this
package only marshals torch tensors into those calls (capi.py) and wraps them for use from
PyTorch (solver.py), including an autograd Function for the data-term gradient.
Importing the package fails if the library has not been built: there is no CPU fallback.
"""
from . import capi
from .solver import Solver, ScatteredField, scattered_field

__all__ = ["capi", "Solver", "ScatteredField", "scattered_field"]
