"""CPU oracle for the block Jacobi sweeping preconditioner (arXiv 2209.10886).

TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports, links or calls
this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA path: the two
meet only in the seeded input generators of the ``workloads`` package.

Plain complex128 NumPy/SciPy code, written for readability, not speed:

* :mod:`oracle.discretization` - global 5-point operator with first-order
  impedance boundaries (paper Eq. origPbm with T = i*kappa).
* :mod:`oracle.decomposition` - checkerboard partition, the paper's
  multi-index orders and numbering ``m(i, j)`` (Section 2), local
  Robin-coupled problems (Eq. subPbm), liftings (Eq. subPbmLifting) and the
  local scattering / transmission map (Section 3).
* :mod:`oracle.sweeping` - the SGS sweeping preconditioner as the products of
  elementary factors (Proposition 1 and Eq. sgs_preconditioner_forward_backward),
  the block Jacobi sweeping preconditioner (Section 5) and the volume
  preconditioner built from them.
* :mod:`oracle.krylov` - restarted flexible GMRES (right preconditioning,
  modified Gram-Schmidt, dense least squares on the Hessenberg matrix).
* :mod:`oracle.adjoint` - source-receiver misfit and its adjoint-state gradient.
* :mod:`oracle.habc` - the Pade-type high-order transmission operator
  (``Decomposition(..., transmission="habc")``).
* :mod:`oracle.parallel` - the same sweeps with the local solves of a stage run
  in worker processes (the all-cores CPU baseline).

Every function states the passage it follows, and the reading it takes where
the paper is silent or ambiguous.
"""
from .discretization import assemble_operator, ghost_factor, operator_diagonal_derivative
from .decomposition import Decomposition
from .sweeping import Sweeper, schedule_steps
from . import habc
from .krylov import fgmres
from .adjoint import misfit_gradient_direct, misfit_gradient_iterative, misfit_value

__all__ = [
    "assemble_operator",
    "ghost_factor",
    "operator_diagonal_derivative",
    "Decomposition",
    "Sweeper",
    "schedule_steps",
    "fgmres",
    "misfit_gradient_direct",
    "misfit_gradient_iterative",
    "misfit_value",
]
