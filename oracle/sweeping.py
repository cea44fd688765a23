"""Sweeping preconditioners on the interface problem (paper Sections 3-5).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The interface problem (Section 3, Eq. abstractSys) is ``(I - S) g = b``:
``b_(j,i)`` is the outgoing data toward j of the lifting ``w_i`` (local solve
with the true source and zero incoming data, Eq. subPbmLifting), and
``(S x)_(j,i)`` is the outgoing data toward j of the local solve of i with zero
source and incoming data ``x_(i, .)`` on all its sides (local scattering
operator).  Neighbours always lie on adjacent diagonals, so ``S`` has no block
on its block diagonal when the unknowns are grouped by the diagonal of their
first index (the matrices ``V_i`` of Section 4).

``E_d = V_d S_{d,d-1} V_{d-1}^T`` moves data from the subdomains of diagonal
d-1 to the unknowns of diagonal d; ``F_d = V_{d-1} S_{d-1,d} V_d^T`` moves it
back.  Proposition 1: ``S_L = I - sum_d E_d`` and ``S_U = I - sum_d F_d`` are
products of the elementary factors ``(I - E_d)`` / ``(I - F_d)``, so (Eq.
sgs_preconditioner_forward_backward)

    S_L^{-1} = (I + E_{Ng+1}) ... (I + E_3),     S_U^{-1} = (I + F_3) ... (I + F_{Ng+1}),

each factor being one *step*; the SGS sweeping preconditioner is
``S_U^{-1} S_L^{-1}``, 2(Ng-1) steps.

Block Jacobi sweeping (Section 5) restricts the triangular factors to bands of
diagonals ``W_{L,g}``: ``2+(g-1)N1 <= |i|_1 <= 2+g N1`` and ``W_{U,g}``:
``(1+Ng)-g N1 <= |i|_1 <= (1+Ng)-(g-1) N1`` (bounds as printed, inclusive), and
runs the restricted substitutions of all bands concurrently, ``2 N1`` steps.

Readings of the garbled/ambiguous passages of Section 5:
* The block written ``(I_i + S_{L,i})^{-1}`` is read as the inverse of the
  band-restricted unit lower-triangular matrix ``W^T S_L W`` (which already
  contains I): a forward substitution inside the band.
* Consecutive bands share one diagonal.  The additive sum would count that
  diagonal twice; it is read as restricted-additive: the shared diagonal takes
  the value propagated by the band in which it is the last diagonal, and the
  next band uses it only as its unpropagated start.  Symmetrically for the
  backward bands (the value comes from the band above).
* The update is the two half-steps as printed, with the residual recomputed
  between them: ``x' = B_L^{-1} b``, ``rho = b - (I - S) x'``,
  ``x = x' + B_U^{-1} rho`` (starting from ``x^(0) = 0``).  With a single band
  this equals ``S_U^{-1} S_L^{-1} b`` exactly.
"""
from __future__ import annotations

import numpy as np


def bands(N1, Ng, direction, overlap=True):
    """Diagonal ranges ``[lo, hi]`` of the block Jacobi bands (Section 5).

    ``direction='L'``: forward bands from the bottom-left corner; ``'U'``:
    backward bands from the top-right corner.  ``overlap=False`` gives the
    non-overlapping variant (bands of N1 diagonals that share none).
    """
    out = []
    g = 1
    lo_all, hi_all = 2, Ng + 1
    width = N1 if overlap else N1 - 1
    while True:
        if direction == "L":
            lo = 2 + (g - 1) * (width + (0 if overlap else 1))
            hi = lo + width
        else:
            hi = (1 + Ng) - (g - 1) * (width + (0 if overlap else 1))
            lo = hi - width
        lo, hi = max(lo, lo_all), min(hi, hi_all)
        if lo > hi_all or hi < lo_all:
            break
        out.append((lo, hi))
        if (direction == "L" and hi >= hi_all) or (direction == "U" and lo <= lo_all):
            break
        g += 1
    return out


def schedule_steps(N1, N2, kind, overlap=True):
    """Sequential steps per preconditioner application: SP ``2(Ng-1)`` (Section 4),
    BSP ``2 x`` the longest band (``2 N1`` when there are at least two bands, Section 5)."""
    Ng = N1 + N2 - 1
    if kind == "SP":
        return 2 * (Ng - 1)
    fw = max(hi - lo for lo, hi in bands(N1, Ng, "L", overlap))
    bw = max(hi - lo for lo, hi in bands(N1, Ng, "U", overlap))
    return fw + bw


class Sweeper:
    """Interface-level operators and preconditioners on one :class:`Decomposition`."""

    def __init__(self, dec):
        self.dec = dec
        self.steps = 0      # sequential steps taken by the last sweep
        self.interface_steps = 0   # interface Krylov steps of precondition_interface_krylov, summed

    # ------------------------------------------------------------- S and E, F
    def scatter_from(self, i, x):
        """Local solve of i with zero source and incoming ``x_(i,.)``; returns
        ``{j: outgoing toward j}`` (one block column of S)."""
        dec = self.dec
        inc = dec.incoming_of(x, i)
        u = dec.local_solve(i, None, inc)
        return {j: dec.outgoing(i, j, u, inc[j]) for j in dec.neighbours(i)}

    def apply_S(self, x):
        """``S x`` over all subdomains (the interface operator of Eq. abstractSys)."""
        y = self.dec.zero_trace()
        for i in self.dec.subdomains:
            for j, v in self.scatter_from(i, x).items():
                y[(j, i)] = v
        return y

    def apply_elementary(self, x, d, kind, restrict=None):
        """In place: ``x <- (I + E_d) x`` (kind 'E': from diagonal d-1 into d) or
        ``x <- (I + F_d) x`` (kind 'F': from diagonal d into d-1).

        ``restrict``: optional set of diagonals the factor is restricted to (the
        band matrices ``W^T . W`` of Section 5); only unknowns whose first index
        lies in that set are read or written.
        """
        dec = self.dec
        src_d, dst_d = (d - 1, d) if kind == "E" else (d, d - 1)
        if restrict is not None and (src_d not in restrict or dst_d not in restrict):
            return
        for i in dec.on_diagonal(src_d):
            outs = self.scatter_from(i, x)
            for j, v in outs.items():
                if dec.diagonal(j) == dst_d:
                    x[(j, i)] = x[(j, i)] + v

    # ------------------------------------------------------------------ SGS / SP
    def inv_SL(self, b, restrict=None, diags=None):
        """``S_L^{-1} b = (I + E_{Ng+1}) ... (I + E_3) b`` (E_3 applied first)."""
        Ng = self.dec.Ng
        x = {k: v.copy() for k, v in b.items()}
        ds = range(3, Ng + 2) if diags is None else diags
        for d in ds:
            self.apply_elementary(x, d, "E", restrict)
        return x

    def inv_SU(self, b, restrict=None, diags=None):
        """``S_U^{-1} b = (I + F_3) ... (I + F_{Ng+1}) b`` (F_{Ng+1} applied first)."""
        Ng = self.dec.Ng
        x = {k: v.copy() for k, v in b.items()}
        ds = range(Ng + 1, 2, -1) if diags is None else diags
        for d in ds:
            self.apply_elementary(x, d, "F", restrict)
        return x

    def sgs(self, b):
        """SGS sweeping preconditioner ``P_SGS^{-1} b = S_U^{-1} S_L^{-1} b`` (Section 4)."""
        self.steps = 2 * (self.dec.Ng - 1)
        return self.inv_SU(self.inv_SL(b))

    # ------------------------------------------------------------ block Jacobi
    def _restrict_vec(self, x, diags):
        dec = self.dec
        return {ij: (v.copy() if dec.diagonal(ij[0]) in diags else np.zeros_like(v))
                for ij, v in x.items()}

    def block_jacobi_L(self, b, overlap=True):
        """``B_L^{-1} b``: band-restricted forward substitutions, restricted-additive combination."""
        dec = self.dec
        out = dec.zero_trace()
        Ng = dec.Ng
        for g, (lo, hi) in enumerate(bands(dec.N1, Ng, "L", overlap)):
            band = set(range(lo, hi + 1))
            xg = self.inv_SL(self._restrict_vec(b, band), restrict=band, diags=range(lo + 1, hi + 1))
            own = set(range(lo + 1, hi + 1)) | ({lo} if g == 0 or not overlap else set())
            for ij in dec.slots:
                if dec.diagonal(ij[0]) in own:
                    out[ij] = xg[ij]
        return out

    def block_jacobi_U(self, r, overlap=True):
        """``B_U^{-1} r``: band-restricted backward substitutions, restricted-additive combination."""
        dec = self.dec
        out = dec.zero_trace()
        Ng = dec.Ng
        for g, (lo, hi) in enumerate(bands(dec.N1, Ng, "U", overlap)):
            band = set(range(lo, hi + 1))
            yg = self.inv_SU(self._restrict_vec(r, band), restrict=band, diags=range(hi, lo, -1))
            own = set(range(lo, hi)) | ({hi} if g == 0 or not overlap else set())
            for ij in dec.slots:
                if dec.diagonal(ij[0]) in own:
                    out[ij] = yg[ij]
        return out

    def bsp(self, b, overlap=True):
        """Block Jacobi sweeping preconditioner (Section 5), one application from ``x^(0) = 0``:
        ``x' = B_L^{-1} b``, ``rho = b - (I - S) x'``, ``x = x' + B_U^{-1} rho``."""
        dec = self.dec
        self.steps = schedule_steps(dec.N1, dec.N2, "BSP", overlap)
        xh = self.block_jacobi_L(b, overlap)
        Sx = self.apply_S(xh)
        rho = {ij: b[ij] - xh[ij] + Sx[ij] for ij in dec.slots}
        y = self.block_jacobi_U(rho, overlap)
        return {ij: xh[ij] + y[ij] for ij in dec.slots}

    # --------------------------------------------------------- volume operator
    def lifting_traces(self, r):
        """``b``: outgoing data of the liftings ``w_i`` (local solves with source r, zero incoming)."""
        dec = self.dec
        b = dec.zero_trace()
        for i in dec.subdomains:
            w = dec.local_solve(i, dec.restrict(r, i), {})
            for j in dec.neighbours(i):
                b[(j, i)] = dec.outgoing(i, j, w, np.zeros(dec.side_length(i, j)))
        return b

    def reconstruct(self, r, g):
        """Volume field: local solves with source r and incoming data g on every subdomain."""
        dec = self.dec
        z = np.zeros(dec.n * dec.n, dtype=np.complex128)
        for i in dec.subdomains:
            u = dec.local_solve(i, dec.restrict(r, i), dec.incoming_of(g, i))
            dec.insert(z, i, u)
        return z

    def precondition(self, r, kind="BSP", overlap=True):
        """Volume preconditioner ``z = M^{-1} r`` (r in the units of the scaled rows):
        liftings -> interface right-hand side b -> ``g ~ (I - S)^{-1} b`` by the
        chosen sweep -> local reconstruction.  With the exact interface solve,
        ``M^{-1} = A^{-1}``."""
        b = self.lifting_traces(r)
        if kind == "SP":
            g = self.sgs(b)
        elif kind == "BSP":
            g = self.bsp(b, overlap)
        elif kind == "exact":
            g = self.exact_interface_solve(b)
        else:
            raise ValueError(kind)
        return self.reconstruct(r, g)

    def precondition_interface_krylov(self, r, kind="BSP", tol=1e-4, restart=100, maxit=100):
        """Volume preconditioner with the interface problem solved iteratively: the
        paper's own use of the sweeps (Sections 3-5), GMRES on ``(I - S) g = b``
        preconditioned by one SP or BSP application, here flexible GMRES to a
        relative residual ``tol`` (at most ``maxit`` steps, restart ``restart``)
        between the liftings and the reconstruction.  As ``tol -> 0`` this tends
        to the exact interface solve, i.e. ``M^{-1} = A^{-1}``."""
        from .krylov import fgmres
        dec = self.dec
        b = dec.flatten(self.lifting_traces(r))
        sweep = self.sgs if kind == "SP" else self.bsp

        def interface_operator(v):
            return v - dec.flatten(self.apply_S(dec.unflatten(v)))

        def interface_precond(v):
            return dec.flatten(sweep(dec.unflatten(v)))

        g, it, _ = fgmres(interface_operator, interface_precond, b, tol=tol, restart=restart, maxit=maxit)
        self.interface_steps += it          # running count of interface Krylov steps (bookkeeping only)
        return self.reconstruct(r, dec.unflatten(g))

    # ------------------------------------------------------------ dense (tiny)
    def dense_S(self):
        """Dense matrix of S in the numbering m(i, j) (tiny problems only)."""
        dec = self.dec
        L = sum(dec.side_length(*ij) for ij in dec.slots)
        S = np.zeros((L, L), dtype=np.complex128)
        for k in range(L):
            e = np.zeros(L, dtype=np.complex128)
            e[k] = 1.0
            S[:, k] = dec.flatten(self.apply_S(dec.unflatten(e)))
        return S

    def exact_interface_solve(self, b):
        dec = self.dec
        S = self.dense_S()
        g = np.linalg.solve(np.eye(S.shape[0]) - S, dec.flatten(b))
        return dec.unflatten(g)
