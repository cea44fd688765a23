"""Global discretisation of the model problem (paper Section 3, Eq. origPbm).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's model problem is ``(-Delta - kappa^2) u = 0`` in the domain with
``(d_n - T) u = 0`` on the artificial boundary, time dependence ``e^{-i w t}``.
This build takes the basic impedance operator ``T = i kappa`` (the paper's
Section 3 uses it for the algebra) and adds a volume source ``f``:

    (-Delta - kappa^2) u = f   in (0,1)^2,      d_n u - i kappa u = 0  on the boundary.

Five-point finite differences on the n x n interior nodes ``x_{a,b} = (a h, b h)``
(h = 1/(n+1)), every row multiplied by h^2:

    4 u_p - sum_{grid neighbours q} u_q - (kappa_p h)^2 u_p - sum_{outer ghost sides} c_p u_p = h^2 f_p

Reading (the paper uses finite elements and says nothing about FD): the
boundary condition is imposed at the mid-edge between the boundary node p and
a ghost node outside, ``(u_gh - u_p)/h - i kappa_p (u_gh + u_p)/2 = 0``, which
gives ``u_gh = c_p u_p`` with ``c_p = (1 + beta_p)/(1 - beta_p)`` and
``beta_p = i kappa_p h / 2``.  A corner node has two ghost sides.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def ghost_factor(beta):
    """Ratio ``u_ghost / u_p`` that makes the mid-edge impedance condition hold.

    From ``(u_gh - u_p)/h - i kappa (u_gh + u_p)/2 = 0`` with ``beta = i kappa h/2``:
    ``u_gh (1 - beta) = u_p (1 + beta)``.
    """
    return (1.0 + beta) / (1.0 - beta)


def node_coordinates(n):
    """0-based (a, b) index arrays of the flat node ordering (y slowest)."""
    a = np.tile(np.arange(n), n)
    b = np.repeat(np.arange(n), n)
    return a, b


def outer_ghost_count(n):
    """Number of sides of each node that face the outer boundary (0, 1 or 2)."""
    a, b = node_coordinates(n)
    return ((a == 0).astype(int) + (a == n - 1) + (b == 0) + (b == n - 1))


def assemble_operator(n, h, omega, m2):
    """The h^2-scaled global matrix A (scipy CSR, complex128), row p as in the module docstring.

    ``m2`` is the squared slowness; ``kappa_p = omega sqrt(m2_p)``.
    """
    m2 = np.asarray(m2, dtype=np.float64)
    N = n * n
    kappa = omega * np.sqrt(m2)
    beta = 0.5j * kappa * h
    diag = 4.0 - (kappa * h) ** 2 - outer_ghost_count(n) * ghost_factor(beta)
    a, _ = node_coordinates(n)
    east = np.where(a[:-1] < n - 1, -1.0, 0.0)     # coupling p -> p+1 only inside a grid row
    north = -np.ones(N - n)
    A = sp.diags([diag, east, east, north, north], [0, 1, -1, n, -n], shape=(N, N), format="csr",
                 dtype=np.complex128)
    A.eliminate_zeros()
    return A


def operator_diagonal_derivative(n, h, omega, m2):
    """``dA_pp / d m2_p`` of the h^2-scaled matrix (A depends on m2 only through its diagonal).

    ``A_pp = 4 - omega^2 h^2 m2_p - n_ghost(p) c(beta_p)`` with ``beta_p = i omega h sqrt(m2_p)/2``;
    ``dc/dbeta = 2/(1-beta)^2`` and ``dbeta/dm2 = i omega h / (4 sqrt(m2))``.
    """
    m2 = np.asarray(m2, dtype=np.float64)
    beta = 0.5j * omega * np.sqrt(m2) * h
    dbeta = 1j * omega * h / (4.0 * np.sqrt(m2))
    return -(omega * h) ** 2 - outer_ghost_count(n) * (2.0 / (1.0 - beta) ** 2) * dbeta


def nested_dissection_order(nx, ny, leaf=64):
    """A fill-reducing ordering of the nx x ny grid (flat index b*nx + a): the two
    halves of the longer side first (recursively), then the grid line that separates
    them, down to boxes of at most ``leaf`` nodes (George's nested dissection).  A
    permutation of 0..nx*ny-1; it changes the cost of the sparse LU, not the system."""
    order = []

    def box(x0, x1, y0, y1):
        w, h = x1 - x0, y1 - y0
        if w <= 0 or h <= 0:
            return
        if w * h <= leaf:
            for b in range(y0, y1):
                order.extend(range(b * nx + x0, b * nx + x1))
            return
        if w >= h:
            m = (x0 + x1) // 2
            box(x0, m, y0, y1)
            box(m + 1, x1, y0, y1)
            order.extend(b * nx + m for b in range(y0, y1))
        else:
            m = (y0 + y1) // 2
            box(x0, x1, y0, m)
            box(x0, x1, m + 1, y1)
            order.extend(range(m * nx + x0, m * nx + x1))

    box(0, nx, 0, ny)
    return np.asarray(order, dtype=np.int64)


class GridDirectSolver:
    """``A^{-1} b`` for a matrix on the n x n grid by a sparse LU (scipy ``splu``) of the
    symmetrically permuted matrix ``A[p][:, p]`` with the nested-dissection order p,
    followed by iterative refinement with the unpermuted A.  The same solution as
    ``spsolve(A, b)`` (the permutation is exact); the order only makes the 10^6-unknown
    systems of the workloads factor in seconds instead of minutes."""

    def __init__(self, A, n, refine=2):
        import scipy.sparse.linalg as spla
        self.A = A.tocsr()
        self.p = nested_dissection_order(n, n)
        Ap = A.tocsc()[self.p][:, self.p].tocsc()
        self.lu = spla.splu(Ap, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                            options=dict(SymmetricMode=True))
        self.refine = refine

    def _raw(self, b):
        x = np.empty_like(b)
        x[self.p] = self.lu.solve(b[self.p])
        return x

    def solve(self, b):
        b = np.asarray(b, dtype=np.complex128)
        x = self._raw(b)
        for _ in range(self.refine):
            x = x + self._raw(b - self.A @ x)
        return x
