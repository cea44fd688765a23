"""Source-receiver misfit and its adjoint-state gradient.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no inverse problem; this is the differentiation workload built
on top of its forward solver.  For sources ``f_s`` the fields solve the scaled
system ``A(m2) u_s = h^2 f_s`` (oracle.discretization).  With the receiver
sampling ``P`` (rows of the identity at the receiver nodes) and data ``d_s``:

    J(m2) = 1/2 sum_s || P u_s - d_s ||^2

Adjoint-state method: ``A^H lambda_s = P^T (P u_s - d_s)`` and, since A
depends on m2 only through its diagonal,

    dJ/dm2_p = - sum_s Re( conj(lambda_{s,p}) (dA_pp/dm2_p) u_{s,p} ).

A is complex symmetric, so ``lambda_s = conj(A^{-1} conj(P^T (P u_s - d_s)))``:
the adjoint solve reuses the forward operator and preconditioner.  The
interface wavenumbers ``kappa_e`` of the decomposition do not change the
discrete solution, so they contribute no term.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .discretization import assemble_operator, operator_diagonal_derivative


def misfit_value(n, h, omega, m2, F, rec, d):
    """J(m2) by direct solves (F: (nsrc, N) sources, unscaled)."""
    A = assemble_operator(n, h, omega, m2).tocsc()
    lu = spla.splu(A)
    J = 0.0
    for s in range(F.shape[0]):
        u = lu.solve(h * h * F[s])
        J += 0.5 * np.sum(np.abs(u[rec] - d[s]) ** 2)
    return J


def misfit_gradient_direct(n, h, omega, m2, F, rec, d):
    """(J, grad, U) with forward and adjoint solves by a sparse direct solver."""
    A = assemble_operator(n, h, omega, m2).tocsc()
    lu = spla.splu(A)
    luH = spla.splu(A.conj().T.tocsc())
    da = operator_diagonal_derivative(n, h, omega, m2)
    J = 0.0
    grad = np.zeros(n * n)
    U = np.zeros_like(F, dtype=np.complex128)
    for s in range(F.shape[0]):
        u = lu.solve(h * h * F[s])
        U[s] = u
        res = u[rec] - d[s]
        J += 0.5 * np.sum(np.abs(res) ** 2)
        r = np.zeros(n * n, dtype=np.complex128)
        r[rec] = res
        lam = luH.solve(r)                         # A^H lambda = P^T (P u - d)
        grad -= np.real(np.conj(lam) * da * u)
    return J, grad, U


def misfit_gradient_iterative(n, h, omega, m2, F, rec, d, solve):
    """Same quantities with a user-supplied solver ``solve(rhs) -> A^{-1} rhs``
    (e.g. FGMRES with the sweeping preconditioner).  The adjoint uses
    ``lambda = conj(A^{-1} conj(P^T (P u - d)))`` (A complex symmetric)."""
    da = operator_diagonal_derivative(n, h, omega, m2)
    J = 0.0
    grad = np.zeros(n * n)
    U = np.zeros_like(F, dtype=np.complex128)
    for s in range(F.shape[0]):
        u = solve(h * h * F[s])
        U[s] = u
        res = u[rec] - d[s]
        J += 0.5 * np.sum(np.abs(res) ** 2)
        r = np.zeros(n * n, dtype=np.complex128)
        r[rec] = res
        lam = np.conj(solve(np.conj(r)))
        grad -= np.real(np.conj(lam) * da * u)
    return J, grad, U
