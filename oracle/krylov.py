"""Restarted flexible GMRES (the paper's Krylov solver, Section 6).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper runs GMRES to a relative residual of 1e-6.  With a preconditioner
that is itself an approximate solve the flexible variant is used (right
preconditioning; the preconditioned directions ``z_j`` are stored and the
update is ``x += Z y``).  This oracle is written for clarity: modified
Gram-Schmidt Arnoldi and, at every step, the small least-squares problem
``min_y || beta e_1 - H y ||`` solved by ``numpy.linalg.lstsq`` (which is the
definition of the GMRES iterate), instead of Givens rotations.
"""
from __future__ import annotations

import numpy as np


def fgmres(matvec, precond, b, tol=1e-6, restart=50, maxit=1000, x0=None, history=None):
    """Solve ``A x = b``; returns ``(x, iterations, true_relative_residual)``.

    ``matvec(v)`` applies A, ``precond(v)`` applies the (possibly varying)
    right preconditioner.  Stops when the true relative residual
    ``||b - A x|| / ||b||`` (checked at every restart and at exit) is at most
    ``tol``, or after ``maxit`` Arnoldi steps.  ``history`` (a list) receives the
    Arnoldi residual estimate after every step.
    """
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    it = 0
    r = b - matvec(x)
    relres = np.linalg.norm(r) / bnorm
    while relres > tol and it < maxit:
        beta = np.linalg.norm(r)
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        y = np.zeros(0, dtype=np.complex128)
        for j in range(restart):
            Z.append(precond(V[j]))
            w = matvec(Z[j])
            for k in range(j + 1):                      # modified Gram-Schmidt
                H[k, j] = np.vdot(V[k], w)
                w = w - H[k, j] * V[k]
            H[j + 1, j] = np.linalg.norm(w)
            it += 1
            rhs = np.zeros(j + 2, dtype=np.complex128)
            rhs[0] = beta
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], rhs, rcond=None)
            est = np.linalg.norm(rhs - H[: j + 2, : j + 1] @ y) / bnorm
            if history is not None:
                history.append(est)
            if est <= tol or it >= maxit or H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
        for k in range(len(y)):
            x = x + y[k] * Z[k]
        r = b - matvec(x)
        relres = np.linalg.norm(r) / bnorm
    return x, it, relres
