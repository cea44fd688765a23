"""Checkerboard decomposition, local Robin problems and transmission (paper Sections 2-3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation (paper Section 2): a subdomain is a multi-index ``i = (i1, i2)`` with
``i1 = 1..N1`` the column and ``i2 = 1..N2`` the row; ``|i|_1 = i1 + i2`` is its
diagonal.  ``D_i`` is the set of its edge neighbours.  Subdomain (1, 1) is the
bottom-left one (the forward sweep runs from the bottom-left to the top-right
corner, Section 6).

Interface unknowns (Section 3): the unknown ``(i, j)``, ``j in D_i``, is the
incoming Robin data of subdomain ``i`` on the interface it shares with ``j``,
``g_{m(i,j)} = (d_{n_{i,j}} - T) v_i``.  It is a vector with one value per
mid-edge point of that interface, ordered by increasing coordinate along it.

Discrete local problem (Eq. subPbm, five-point stencil, rows scaled by h^2).
Across an interface edge between ``p in Omega_i`` and ``q in Omega_j`` the
ghost value of subdomain ``i`` satisfies, at the mid-edge, the Robin condition
``(d_n - T_e) u = g``:

    (u_gh - u_p)/h - T_e (u_p + u_gh)/2 = g_{i<-j}

so with ``G = h g`` and ``beta_e = T_e h/2``:
``u_gh = (G + (1 + beta_e) u_p)/(1 - beta_e)``.  Substituting into the stencil
row of ``p`` moves ``(1+beta_e)/(1-beta_e) u_p`` to the diagonal and
``G/(1-beta_e)`` to the right-hand side.  The outer boundary keeps the
first-order absorbing condition ``T = i kappa_p`` (Eq. origPbm).

Readings taken where the paper (finite elements, Pade HABC) says nothing:
* ``kappa_e = omega sqrt((m2_p + m2_q)/2)``, the same value seen from both sides.
* The outgoing data toward ``j``, ``(-d_{n_{i,j}} - T) u_i`` (Eq. subPbm), is
  ``-G_in - 2 T_e h (u_p + u_gh)/2`` in scaled form, i.e.
  ``G_out = -((1 + beta_e) G_in + 4 beta_e u_p)/(1 - beta_e)``.
* The interface operator ``T_e`` (see :meth:`Decomposition.transmission_operator`)
  is either the basic impedance ``i kappa_e`` the paper uses for its algebra
  (Section 3) or an optimized complex Robin parameter.  Any ``T_e`` common to
  both sides of an edge leaves the converged solution unchanged (the
  decomposition is consistent with the global rows); only the convergence of
  the sweeps depends on it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import habc
from .discretization import ghost_factor


def ghost_matrix(B):
    """``(I - B)^{-1} (I + B)``: the ghost values ``u_g = C u_p`` of one side when its
    condition ``(u_g - u_p)/h - T (u_g + u_p)/2 = 0`` has a matrix ``B = T h / 2``
    (the scalar :func:`ghost_factor` along the side's points when B is diagonal)."""
    Id = np.eye(B.shape[0], dtype=np.complex128)
    return np.linalg.solve(Id - B, Id + B)

# sides of a subdomain, named by the direction of the neighbour
WEST, EAST, SOUTH, NORTH = "W", "E", "S", "N"


def multi_index_key(i):
    """Sort key of the paper's order on multi-indices (Section 2, first definition):
    ``i < j`` iff ``|i|_1 < |j|_1``, or ``|i|_1 = |j|_1`` and ``i1 < j1``."""
    return (i[0] + i[1], i[0])


def pair_key(i, j):
    """Sort key of the order on pairs (Section 2, second definition):
    ``(i, j) < (k, l)`` iff ``i < k``, or ``i = k`` and ``j < l``."""
    return multi_index_key(i) + multi_index_key(j)


class Decomposition:
    """A checkerboard partition of the n x n grid with its local problems.

    ``xcuts``/``ycuts`` are node offsets (length N1+1 / N2+1).  Column ``i1``
    owns 0-based x-nodes ``xcuts[i1-1] .. xcuts[i1]-1``.
    """

    def __init__(self, n, h, omega, m2, xcuts, ycuts, transmission="optimized", tc_scale=1.0,
                 n_pade=8, phi=np.pi / 3):
        self.n, self.h, self.omega = n, h, omega
        self.transmission, self.tc_scale = transmission, tc_scale
        self.n_pade, self.phi = n_pade, phi         # transmission = "habc" (oracle.habc)
        self.m2 = np.asarray(m2, dtype=np.float64).reshape(n, n)   # [b, a]
        self.xcuts = [int(v) for v in xcuts]
        self.ycuts = [int(v) for v in ycuts]
        self.N1 = len(self.xcuts) - 1
        self.N2 = len(self.ycuts) - 1
        # Section 2: N_dom, N_e, N_g
        self.Ndom = self.N1 * self.N2
        self.Ne = 2 * self.N1 * self.N2 - self.N1 - self.N2
        self.Ng = self.N1 + self.N2 - 1
        self.subdomains = sorted(
            [(i1, i2) for i1 in range(1, self.N1 + 1) for i2 in range(1, self.N2 + 1)],
            key=multi_index_key)
        self._lu = {}
        self._mat = {}
        self._edges = {}
        for i in self.subdomains:
            for j in self.neighbours(i):
                self._edges[(i, j)] = self._edge_geometry(i, j)
        # the paper's numbering m(i, j): position of the pair in the pair order, from 1
        self.slots = sorted(self._edges.keys(), key=lambda ij: pair_key(*ij))
        assert len(self.slots) == 2 * self.Ne
        self.m = {ij: k + 1 for k, ij in enumerate(self.slots)}

    # ----------------------------------------------------------------- geometry
    def box(self, i):
        """Half-open node box ``(x0, x1, y0, y1)`` of subdomain i (0-based)."""
        i1, i2 = i
        return self.xcuts[i1 - 1], self.xcuts[i1], self.ycuts[i2 - 1], self.ycuts[i2]

    def diagonal(self, i):
        """``|i|_1``, in 2..Ng+1."""
        return i[0] + i[1]

    def on_diagonal(self, d):
        return [i for i in self.subdomains if self.diagonal(i) == d]

    def neighbours(self, i):
        """``D_i``: edge neighbours of i inside the N1 x N2 lattice."""
        i1, i2 = i
        out = []
        for j in ((i1 - 1, i2), (i1 + 1, i2), (i1, i2 - 1), (i1, i2 + 1)):
            if 1 <= j[0] <= self.N1 and 1 <= j[1] <= self.N2:
                out.append(j)
        return out

    def side(self, i, j):
        di = (j[0] - i[0], j[1] - i[1])
        return {(-1, 0): WEST, (1, 0): EAST, (0, -1): SOUTH, (0, 1): NORTH}[di]

    def _edge_geometry(self, i, j):
        """Own boundary nodes ``p`` (flat local indices), the neighbour's nodes ``q``
        (global (b, a)) and ``beta_e`` along the interface of i facing j."""
        x0, x1, y0, y1 = self.box(i)
        mx = x1 - x0
        s = self.side(i, j)
        if s in (WEST, EAST):
            ys = np.arange(y0, y1)
            ap = x0 if s == WEST else x1 - 1
            aq = ap - 1 if s == WEST else ap + 1
            p_local = (ys - y0) * mx + (ap - x0)
            mp, mq = self.m2[ys, ap], self.m2[ys, aq]
        else:
            xs = np.arange(x0, x1)
            bp = y0 if s == SOUTH else y1 - 1
            bq = bp - 1 if s == SOUTH else bp + 1
            p_local = (bp - y0) * mx + (xs - x0)
            mp, mq = self.m2[bp, xs], self.m2[bq, xs]
        kappa_e = self.omega * np.sqrt(0.5 * (mp + mq))
        if self.transmission == "habc":
            # beta_e = T h / 2 as the side's dense matrix (oracle.habc)
            return p_local, 0.5 * self.h * habc.side_operator(kappa_e, self.h, self.n_pade, self.phi)
        beta_e = 0.5 * self.h * self.transmission_operator(kappa_e)
        return p_local, beta_e

    def transmission_operator(self, kappa_e):
        """Robin parameter ``T_e`` of the interface condition ``(d_n - T_e) u = g``.

        ``'impedance'``: ``T_e = i kappa_e``, the basic impedance operator of
        the paper's Section 3.  Its reflection coefficient has modulus one for
        evanescent modes, and restarted Krylov stagnates on fine grids.
        ``'optimized'``: ``T_e = (i - 1) p0`` with
        ``p0 = s sqrt(kappa_e k_max / 2)``, ``k_max = pi/h`` (the largest
        frequency the grid carries), ``s = tc_scale``: a complex Robin
        parameter of the "optimized zeroth-order" form from the optimized
        Schwarz literature (Gander, Magoules, Nataf 2002), whose negative real
        part damps evanescent modes and whose imaginary part passes
        propagating ones.
        """
        if self.transmission == "impedance":
            return 1j * kappa_e
        if self.transmission != "optimized":
            raise ValueError(self.transmission)
        kmax = np.pi / self.h
        p0 = self.tc_scale * np.sqrt(0.5 * kappa_e * kmax)
        return (1j - 1.0) * p0

    def side_length(self, i, j):
        return len(self._edges[(i, j)][0])

    # ------------------------------------------------------------ local problem
    def local_matrix(self, i):
        """Scaled local matrix of Eq. subPbm on the box of i (complex symmetric)."""
        if i in self._mat:
            return self._mat[i]
        x0, x1, y0, y1 = self.box(i)
        mx, my = x1 - x0, y1 - y0
        n, h = self.n, self.h
        m2 = self.m2[y0:y1, x0:x1]
        kappa = self.omega * np.sqrt(m2)
        diag = (4.0 - (kappa * h) ** 2).astype(np.complex128)
        c_outer = ghost_factor(0.5j * kappa * h)
        # outer-boundary sides: ghost factor with the node's own kappa
        if x0 == 0:
            diag[:, 0] -= c_outer[:, 0]
        if x1 == n:
            diag[:, -1] -= c_outer[:, -1]
        if y0 == 0:
            diag[0, :] -= c_outer[0, :]
        if y1 == n:
            diag[-1, :] -= c_outer[-1, :]
        diag = diag.reshape(-1)
        # interface sides: ghost factor with the edge's kappa_e (a dense block for the HABC)
        blocks = []
        for j in self.neighbours(i):
            p_local, beta_e = self._edges[(i, j)]
            if np.ndim(beta_e) == 2:
                blocks.append((p_local, ghost_matrix(beta_e)))
            else:
                np.add.at(diag, p_local, -ghost_factor(beta_e))
        M = mx * my
        la = np.tile(np.arange(mx), my)
        east = np.where(la[:-1] < mx - 1, -1.0, 0.0)
        north = -np.ones(M - mx)
        A = sp.diags([diag, east, east, north, north], [0, 1, -1, mx, -mx], shape=(M, M),
                     format="csc", dtype=np.complex128)
        for p_local, C in blocks:
            rows = np.repeat(p_local, len(p_local))
            cols = np.tile(p_local, len(p_local))
            A = A - sp.csc_matrix((C.reshape(-1), (rows, cols)), shape=(M, M))
        A = A.tocsc()
        self._mat[i] = A
        return A

    def local_solver(self, i):
        """Sparse direct factorisation of the local matrix (the paper solves the
        sub-problems with a sparse direct solver, Section 6)."""
        if i not in self._lu:
            self._lu[i] = spla.splu(self.local_matrix(i))
        return self._lu[i]

    def restrict(self, v, i):
        """Values of a global vector on the nodes of i, local order (y slowest)."""
        x0, x1, y0, y1 = self.box(i)
        return np.asarray(v).reshape(self.n, self.n)[y0:y1, x0:x1].reshape(-1)

    def local_solve(self, i, source, incoming):
        """Solve the local problem of i.

        ``source``: local right-hand side values (already scaled like the rows),
        or None for a zero volume source.  ``incoming``: dict ``j -> G`` of
        scaled incoming data on the interface facing j (missing sides: zero).
        The right-hand side is ``source + sum_j G_j/(1 - beta_e)`` at the
        boundary nodes of each side.
        """
        x0, x1, y0, y1 = self.box(i)
        M = (x1 - x0) * (y1 - y0)
        rhs = np.zeros(M, dtype=np.complex128) if source is None else np.array(source, dtype=np.complex128)
        for j, G in incoming.items():
            p_local, beta_e = self._edges[(i, j)]
            if np.ndim(beta_e) == 2:
                np.add.at(rhs, p_local, np.linalg.solve(np.eye(len(p_local)) - beta_e, G))
            else:
                np.add.at(rhs, p_local, G / (1.0 - beta_e))
        return self.local_solver(i).solve(rhs)

    def outgoing(self, i, j, u_local, G_in):
        """Outgoing data of i toward j, i.e. the incoming data of j from i
        (Eq. subPbm right-hand side ``(-d_{n_{i,j}} - T) u_i``), scaled form:
        ``-((1 + beta_e) G_in + 4 beta_e u_p)/(1 - beta_e)``."""
        p_local, beta_e = self._edges[(i, j)]
        if np.ndim(beta_e) == 2:
            # the same relation with the side matrix B = T h / 2: the ghost values
            # u_g = (I - B)^{-1} ((I + B) u_p + G_in), mid-edge mean m = (u_g + u_p)/2,
            # G_out = -G_in - 4 B m (the scalar formula above when B = beta I)
            B = beta_e
            up = u_local[p_local]
            ug = np.linalg.solve(np.eye(len(up)) - B, up + B @ up + G_in)
            return -G_in - 2.0 * (B @ (ug + up))
        return -((1.0 + beta_e) * G_in + 4.0 * beta_e * u_local[p_local]) / (1.0 - beta_e)

    def insert(self, z, i, u_local):
        """Write local values of i into the global vector z (in place)."""
        x0, x1, y0, y1 = self.box(i)
        z.reshape(self.n, self.n)[y0:y1, x0:x1] = u_local.reshape(y1 - y0, x1 - x0)

    # ------------------------------------------------------ interface vectors
    def zero_trace(self):
        """An interface vector: dict ``(i, j) -> array`` over all 2 N_e unknowns."""
        return {ij: np.zeros(self.side_length(*ij), dtype=np.complex128) for ij in self.slots}

    def incoming_of(self, x, i):
        return {j: x[(i, j)] for j in self.neighbours(i)}

    def flatten(self, x):
        """Concatenate an interface vector in the paper's numbering m(i, j)."""
        return np.concatenate([x[ij] for ij in self.slots])

    def unflatten(self, v):
        out, k = {}, 0
        for ij in self.slots:
            L = self.side_length(*ij)
            out[ij] = np.array(v[k:k + L], dtype=np.complex128)
            k += L
        return out
