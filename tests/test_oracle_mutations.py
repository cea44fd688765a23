"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each test patches one plausible error into the oracle - a dropped term, a
wrong sign, a wrong order or index - and checks that the pin covering that
part fails.  This shows the pins are not vacuous.
"""
import math

import numpy as np
import scipy.sparse.linalg as spla
import scipy.special as ss

import oracle.decomposition as odec
import oracle.discretization as odis
import oracle.sweeping as oswp
import workloads as W
from oracle import Decomposition, Sweeper, assemble_operator


def _exact_interface_error():
    w = W.workload("custom", n=30, N1=3, N2=2, medium="layered", seed=2,
                   xcuts=[0, 11, 19, 30], ycuts=[0, 13, 30])
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    r = W.random_complex(w.N, 11)
    z = Sweeper(dec).precondition(r, "exact")
    u = spla.spsolve(A.tocsc(), r)
    return np.linalg.norm(z - u) / np.linalg.norm(u)


def test_pin_holds_unpatched():
    assert _exact_interface_error() < 1e-12


def test_dropped_incoming_term_in_transmission_is_caught(monkeypatch):
    def bad(self, i, j, u_local, G_in):
        p_local, beta_e = self._edges[(i, j)]
        return -(4.0 * beta_e * u_local[p_local]) / (1.0 - beta_e)
    monkeypatch.setattr(odec.Decomposition, "outgoing", bad)
    assert _exact_interface_error() > 1e-3


def test_wrong_sign_in_transmission_is_caught(monkeypatch):
    def bad(self, i, j, u_local, G_in):
        p_local, beta_e = self._edges[(i, j)]
        return -((1.0 + beta_e) * G_in - 4.0 * beta_e * u_local[p_local]) / (1.0 - beta_e)
    monkeypatch.setattr(odec.Decomposition, "outgoing", bad)
    assert _exact_interface_error() > 1e-3


def test_unscaled_incoming_data_in_local_rhs_is_caught(monkeypatch):
    orig = odec.Decomposition.local_solve

    def bad(self, i, source, incoming):
        # forgets the 1/(1 - beta_e) factor of the incoming data
        x0, x1, y0, y1 = self.box(i)
        M = (x1 - x0) * (y1 - y0)
        rhs = np.zeros(M, dtype=np.complex128) if source is None else np.array(source, dtype=np.complex128)
        for j, G in incoming.items():
            p_local, beta_e = self._edges[(i, j)]
            np.add.at(rhs, p_local, G)
        return self.local_solver(i).solve(rhs)
    monkeypatch.setattr(odec.Decomposition, "local_solve", bad)
    assert _exact_interface_error() > 1e-3
    monkeypatch.setattr(odec.Decomposition, "local_solve", orig)


def test_reversed_sweep_order_is_caught(monkeypatch):
    """Applying the elementary factors of S_L^{-1} in the reverse order is no
    longer a forward substitution: the dense Proposition-1 pin fails."""
    w = W.workload("custom", n=23, N1=3, N2=3, medium="layered", seed=6)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    sw = Sweeper(dec)
    S = sw.dense_S()
    d = np.concatenate([[dec.diagonal(ij[0])] * dec.side_length(*ij) for ij in dec.slots])
    SL = np.eye(len(d)) - np.where(d[:, None] == d[None, :] + 1, S, 0)
    b = dec.unflatten(W.random_complex(len(d), 7))
    ref = np.linalg.solve(SL, dec.flatten(b))
    good = dec.flatten(sw.inv_SL(b))
    bad = dec.flatten(sw.inv_SL(b, diags=range(dec.Ng + 1, 2, -1)))
    assert np.linalg.norm(good - ref) / np.linalg.norm(ref) < 1e-12
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 1e-3


def test_incoming_radiation_sign_is_caught(monkeypatch):
    """Flipping the sign of beta in the outer ABC turns the outgoing condition
    into an incoming one: the Hankel pin fails."""
    orig = odis.ghost_factor
    monkeypatch.setattr(odis, "ghost_factor", lambda beta: orig(-beta))
    n = 255
    h = 1.0 / (n + 1)
    kap = 2 * math.pi / (25 * h)
    A = odis.assemble_operator(n, h, kap, np.ones(n * n)).tocsc()
    c = n // 2
    f = np.zeros(n * n, complex)
    f[c * n + c] = 1.0
    U = spla.spsolve(A, f).reshape(n, n)
    errs = [abs(U[c, c + k] - 0.25j * ss.hankel1(0, kap * k * h)) / abs(0.25j * ss.hankel1(0, kap * k * h))
            for k in (6, 12, 25, 40)]
    assert max(errs) > 0.1


def test_row_major_numbering_is_caught(monkeypatch):
    """Ordering subdomains by (i2, i1) instead of the paper's (|i|_1, i1) breaks
    the paper's example m((1,1),(2,1)) = 2."""
    monkeypatch.setattr(odec, "multi_index_key", lambda i: (i[1], i[0]))
    w = W.workload("custom", n=15, N1=3, N2=3)
    dec = odec.Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    assert dec.m[((1, 1), (2, 1))] != 2 or dec.m[((1, 2), (1, 1))] != 3


def test_double_counted_shared_diagonal_is_caught():
    """The literal additive combination (shared diagonal counted by both bands)
    differs from the restricted-additive reading, which the single-band
    identity BSP == SGS pins."""
    w = W.workload("custom", n=24, N1=2, N2=2, medium="layered", seed=1)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    sw = Sweeper(dec)
    b = dec.unflatten(W.random_complex(sum(dec.side_length(*ij) for ij in dec.slots), 3))
    ref = dec.flatten(sw.sgs(b))
    assert np.linalg.norm(dec.flatten(sw.bsp(b)) - ref) <= 1e-13 * np.linalg.norm(ref)
    # an additive x' that adds b once more on the start diagonal breaks it
    xh = sw.block_jacobi_L(b)
    for ij in dec.slots:
        if dec.diagonal(ij[0]) == 2:
            xh[ij] = xh[ij] + b[ij]
    Sx = sw.apply_S(xh)
    rho = {ij: b[ij] - xh[ij] + Sx[ij] for ij in dec.slots}
    y = sw.block_jacobi_U(rho)
    bad = dec.flatten({ij: xh[ij] + y[ij] for ij in dec.slots})
    assert np.linalg.norm(bad - ref) > 1e-3 * np.linalg.norm(ref)


def _leading_band_error():
    """The first check of the leading-band pin: B_L^{-1} b against S_L^{-1} b on the
    first forward band, for b supported there (2 x 4 checkerboard, three bands)."""
    w = W.workload("custom", n=24, N1=2, N2=4, medium="layered", seed=14)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    sw = Sweeper(dec)
    lo, hi = oswp.bands(dec.N1, dec.Ng, "L")[0]
    full = dec.unflatten(W.random_complex(sum(dec.side_length(*ij) for ij in dec.slots), 12))
    b = {ij: (v.copy() if lo <= dec.diagonal(ij[0]) <= hi else np.zeros_like(v)) for ij, v in full.items()}
    x, ex = sw.block_jacobi_L(b), sw.inv_SL(b)
    sel = [ij for ij in dec.slots if dec.diagonal(ij[0]) <= hi]
    a, e = np.concatenate([x[ij] for ij in sel]), np.concatenate([ex[ij] for ij in sel])
    return np.linalg.norm(a - e) / np.linalg.norm(e)


def test_additive_band_sum_is_caught_by_the_leading_band_pin(monkeypatch):
    """Summing every band's substitution over its whole band (the literal additive
    reading) counts the shared diagonal twice: the leading-band pin fails."""
    assert _leading_band_error() < 1e-13

    def additive_L(self, b, overlap=True):
        dec = self.dec
        out = dec.zero_trace()
        for lo, hi in oswp.bands(dec.N1, dec.Ng, "L", overlap):
            band = set(range(lo, hi + 1))
            xg = self.inv_SL(self._restrict_vec(b, band), restrict=band, diags=range(lo + 1, hi + 1))
            for ij in dec.slots:
                if dec.diagonal(ij[0]) in band:
                    out[ij] = out[ij] + xg[ij]
        return out

    monkeypatch.setattr(oswp.Sweeper, "block_jacobi_L", additive_L)
    assert _leading_band_error() > 1e-3


# ------------------------------------------------ Pade HABC transmission (oracle.habc)
import oracle.habc as ohabc  # noqa: E402


def _habc_fixed_point_error():
    w = W.workload("custom", n=30, N1=3, N2=2, medium="layered", seed=2,
                   xcuts=[0, 11, 19, 30], ycuts=[0, 13, 30])
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission="habc")
    r = W.random_complex(w.N, 11)
    z = Sweeper(dec).precondition(r, "exact")
    u = spla.spsolve(A.tocsc(), r)
    return np.linalg.norm(z - u) / np.linalg.norm(u)


def _neumann_symbol_error():
    L, h, kappa = 21, 0.02, 40.0
    T = ohabc.side_operator(np.full(L, kappa), h, 8, np.pi / 3)
    j = np.arange(L)
    worst = 0.0
    for k in (0, 3, 11):
        v = np.cos(np.pi * k * (j + 0.5) / L)
        lam = -(2.0 - 2.0 * np.cos(np.pi * k / L)) / h ** 2
        sym = 1j * kappa * ohabc.rotated_sqrt(lam / kappa ** 2, 8, np.pi / 3)
        worst = max(worst, np.linalg.norm(T @ v - sym * v) / np.linalg.norm(sym * v))
    return worst


def test_habc_pins_hold_unpatched():
    assert _habc_fixed_point_error() < 1e-12
    assert _neumann_symbol_error() < 1e-10


def test_habc_outgoing_without_the_incoming_term_is_caught(monkeypatch):
    orig = odec.Decomposition.outgoing

    def bad(self, i, j, u_local, G_in):
        return orig(self, i, j, u_local, G_in) + G_in      # drops the -G_in term
    monkeypatch.setattr(odec.Decomposition, "outgoing", bad)
    assert _habc_fixed_point_error() > 1e-3


def test_habc_one_sided_operator_is_caught(monkeypatch):
    """Transposing the side matrix on one side of each interface only breaks the
    fixed point (both sides must apply the same operator)."""
    orig = odec.Decomposition._edge_geometry

    def bad(self, i, j):
        p, B = orig(self, i, j)
        return (p, B.T.copy()) if (np.ndim(B) == 2 and i < j) else (p, B)
    # the layered medium makes kappa_e vary along the side, so B is not symmetric
    monkeypatch.setattr(odec.Decomposition, "_edge_geometry", bad)
    assert _habc_fixed_point_error() > 1e-6


def test_habc_dropped_neumann_ends_are_caught(monkeypatch):
    orig = ohabc.tangential_laplacian

    def bad(L, h):
        D = orig(L, h)
        D[0, 0] -= 1.0 / h ** 2          # Dirichlet instead of Neumann ends
        D[-1, -1] -= 1.0 / h ** 2
        return D
    monkeypatch.setattr(ohabc, "tangential_laplacian", bad)
    assert _neumann_symbol_error() > 1e-3


def test_habc_swapped_pade_coefficients_are_caught(monkeypatch):
    orig = ohabc.pade_coefficients

    def bad(N):
        a, b = orig(N)
        M = 2 * N + 1
        return 2.0 / M * b, a * M / 2.0                 # sin and cos exchanged
    monkeypatch.setattr(ohabc, "pade_coefficients", bad)
    w = 0.1
    err = abs(ohabc.pade_sqrt(w, 3) - np.sqrt(1 + w))
    assert err > 0.05 * w ** 7                          # the Taylor-order pin fails
