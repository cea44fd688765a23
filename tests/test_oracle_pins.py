"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests uses the GPU library.  Each pin is chosen so that a
plausible mistake in the oracle (a dropped term, a wrong sign, a wrong index
or order) makes at least one of them fail; ``test_oracle_mutations.py`` plants
such mistakes and checks that they are caught.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import scipy.special as ss

import workloads as W
from oracle import (Decomposition, Sweeper, assemble_operator, fgmres, ghost_factor,
                    misfit_gradient_direct, misfit_gradient_iterative, misfit_value,
                    operator_diagonal_derivative, schedule_steps)
from oracle.sweeping import bands


def _problem(n, N1, N2, ppw=10.0, medium="const", xcuts=None, ycuts=None, seed=0, nrhs=1,
             transmission="optimized"):
    kw = dict(n=n, N1=N1, N2=N2, ppw=ppw, medium=medium, seed=seed, nrhs=nrhs)
    if xcuts is not None:
        kw["xcuts"] = xcuts
    if ycuts is not None:
        kw["ycuts"] = ycuts
    w = W.workload("custom", **kw)
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission=transmission)
    return w, A, dec, Sweeper(dec)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# --------------------------------------------------------------- discretisation
def test_ghost_factor_satisfies_midedge_impedance():
    """Closed form: u_gh = c u_p makes (u_gh-u_p)/h - i kappa (u_gh+u_p)/2 vanish
    (first-order absorbing condition d_n u - i kappa u = 0, Eq. origPbm with T = i kappa)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        kappa, h, up = rng.uniform(1, 200), rng.uniform(1e-4, 1e-1), rng.normal() + 1j * rng.normal()
        beta = 0.5j * kappa * h
        ugh = ghost_factor(beta) * up
        resid = (ugh - up) / h - 1j * kappa * (ugh + up) / 2
        assert abs(resid) <= 1e-12 * (abs(up) / h)
    # energy: |c| = 1 and Im c > 0 (absorbing for e^{-i w t})
    beta = 0.5j * 0.3
    assert abs(abs(ghost_factor(beta)) - 1) < 1e-15 and ghost_factor(beta).imag > 0


def test_operator_is_complex_symmetric_and_five_point():
    w = W.workload("custom", n=17, N1=1, N2=1, medium="layered", seed=4)
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    assert abs(A - A.T).max() == 0.0
    nnz_rows = np.diff(A.indptr)
    n = w.n
    assert nnz_rows.max() == 5 and nnz_rows.min() == 3      # interior 5, corners 3
    assert A.nnz == 5 * n * n - 4 * n


def test_nested_dissection_solver_is_the_direct_solve():
    """The oracle's fast direct solver (sparse LU of the grid matrix in nested-dissection
    order, plus refinement) is a permutation of the same system: it must return what
    scipy's spsolve returns, on a ragged grid too, and its order must be a permutation."""
    from oracle.discretization import GridDirectSolver, nested_dissection_order
    for n in (1, 5, 17, 40):
        p = nested_dissection_order(n, n)
        assert np.array_equal(np.sort(p), np.arange(n * n))
    w = W.workload("custom", n=45, N1=2, N2=2, medium="layered", seed=6)
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    b = W.random_complex((2, w.N), 12)
    solver = GridDirectSolver(A, w.n)
    for k in range(2):
        assert _rel(solver.solve(b[k]), spla.spsolve(A.tocsc(), b[k])) <= 1e-12


def test_discrete_plane_wave_is_exact():
    """A discrete plane wave solves the interior stencil exactly when
    (kappa h)^2 = 4 - 2 cos(xi h) - 2 cos(eta h); with boundary data built from
    the plane-wave ghost values (not via A) it is the exact discrete solution."""
    n = 41
    h = 1.0 / (n + 1)
    xi, eta = 2 * math.pi * 3.3, -2 * math.pi * 1.7
    kh2 = 4 - 2 * math.cos(xi * h) - 2 * math.cos(eta * h)
    omega = math.sqrt(kh2) / h
    m2 = np.ones(n * n)
    A = assemble_operator(n, h, omega, m2)
    a = np.arange(0, n + 2)                        # 0..n+1 includes ghost positions
    upw = lambda aa, bb: np.exp(1j * (xi * aa * h + eta * bb * h))
    beta = 0.5j * math.sqrt(kh2)
    c = ghost_factor(beta)
    rhs = np.zeros((n, n), dtype=complex)          # h^2 f, [b, a] with 1-based node (a, b)
    for bb in range(1, n + 1):
        for aa in range(1, n + 1):
            s = 0
            for ga, gb in ((aa - 1, bb), (aa + 1, bb), (aa, bb - 1), (aa, bb + 1)):
                if ga in (0, n + 1) or gb in (0, n + 1):
                    s += upw(ga, gb) - c * upw(aa, bb)
            rhs[bb - 1, aa - 1] = s
    u = spla.spsolve(A.tocsc(), rhs.reshape(-1))
    A_, B_ = np.meshgrid(a[1:-1], a[1:-1])
    assert _rel(u, upw(A_, B_).reshape(-1)) < 1e-10


def test_point_source_matches_outgoing_hankel():
    """Loose continuum check of the radiation sign: a unit point source in a
    constant medium at 25 points per wavelength against (i/4) H0^(1)(kappa r),
    the outgoing fundamental solution for e^{-i w t}.  The first-order ABC and
    the FD dispersion leave a few per cent."""
    n = 255
    h = 1.0 / (n + 1)
    kap = 2 * math.pi / (25 * h)
    A = assemble_operator(n, h, kap, np.ones(n * n)).tocsc()
    c = n // 2
    f = np.zeros(n * n, complex)
    f[c * n + c] = 1.0                              # h^2 * (delta / h^2)
    U = spla.spsolve(A, f).reshape(n, n)
    for k in (6, 12, 25, 40):
        ex = 0.25j * ss.hankel1(0, kap * k * h)
        assert abs(U[c, c + k] - ex) / abs(ex) < 0.1
        assert abs(U[c + k, c] - ex) / abs(ex) < 0.1


# ------------------------------------------------------------------ numbering
def test_numbering_matches_paper_example(golden_dir):
    _, _, dec, _ = _problem(15, 3, 3)
    rows = np.loadtxt(os.path.join(golden_dir, "numbering_m.txt"), dtype=int, ndmin=2)
    for i1, i2, j1, j2, m in rows:
        assert dec.m[((i1, i2), (j1, j2))] == m


def test_counts_match_section2():
    for N1, N2 in ((2, 2), (3, 2), (4, 3), (1, 3)):
        _, _, dec, _ = _problem(13, N1, N2)
        assert dec.Ndom == N1 * N2
        assert len(dec.slots) == 2 * (2 * N1 * N2 - N1 - N2)
        assert dec.Ng == N1 + N2 - 1


def test_schedule_steps_match_table1(golden_dir):
    rows = np.loadtxt(os.path.join(golden_dir, "table1_steps.txt"), dtype=int, ndmin=2)
    for N1, N2, sp_ns, bsp_ns in rows:
        assert schedule_steps(N1, N2, "SP") == sp_ns == 2 * (N1 + N2 - 2)
        assert schedule_steps(N1, N2, "BSP") == bsp_ns == 2 * N1
    # 5 x 10 has three partial sweeps ("two cuts", Fig. 3 caption)
    assert len(bands(5, 14, "L")) == 3


# ----------------------------------------------------- DD consistency (exact)
@pytest.mark.parametrize("transmission", ["impedance", "optimized"])
@pytest.mark.parametrize("n,N1,N2,xc,yc", [(31, 2, 2, None, None), (30, 3, 2, [0, 11, 19, 30], [0, 13, 30])])
def test_exact_interface_solve_reproduces_global_solution(n, N1, N2, xc, yc, transmission):
    """With g = (I - S)^{-1} b the local reconstructions equal A^{-1} r exactly:
    the Robin transmission of the decomposition is consistent with the global rows,
    for either interface Robin parameter."""
    w, A, dec, sw = _problem(n, N1, N2, medium="layered", xcuts=xc, ycuts=yc, seed=2,
                             transmission=transmission)
    r = W.random_complex(w.N, 11)
    z = sw.precondition(r, "exact")
    assert _rel(z, spla.spsolve(A.tocsc(), r)) < 1e-12


@pytest.mark.parametrize("kind", ["SP", "BSP"])
def test_interface_krylov_preconditioner_tends_to_the_inverse(kind):
    """GMRES on (I - S) g = b (the paper's formulation) to a tight tolerance gives
    the exact interface solution, so the nested preconditioner reproduces A^{-1} r;
    with a loose tolerance it is a (nonlinear) approximation no better than that."""
    w, A, dec, sw = _problem(30, 3, 2, medium="layered", xcuts=[0, 11, 19, 30], ycuts=[0, 13, 30], seed=2)
    r = W.random_complex(w.N, 17)
    ref = spla.spsolve(A.tocsc(), r)
    z = sw.precondition_interface_krylov(r, kind, tol=1e-13, restart=200, maxit=400)
    assert _rel(z, ref) < 1e-10
    loose = sw.precondition_interface_krylov(r, kind, tol=1e-2, restart=200, maxit=400)
    assert 1e-10 < _rel(loose, ref) < 1.0


def test_single_subdomain_is_a_direct_solve():
    """N1 = N2 = 1: M^{-1} = A^{-1} and FGMRES converges in one iteration."""
    w, A, dec, sw = _problem(33, 1, 1, medium="layered", seed=5)
    r = W.random_complex(w.N, 1)
    assert _rel(sw.precondition(r, "SP"), spla.spsolve(A.tocsc(), r)) < 1e-12
    b = w.h ** 2 * w.f[0]
    x, it, rr = fgmres(lambda v: A @ v, lambda v: sw.precondition(v, "BSP"), b, tol=1e-10)
    assert it == 1 and rr < 1e-10


# ------------------------------------------------------------ sweeps (dense)
def _diag_masks(dec):
    d = np.concatenate([[dec.diagonal(ij[0])] * dec.side_length(*ij) for ij in dec.slots])
    return d


def test_proposition1_and_sgs_products_dense():
    """S_L = I - sum E_d is the product of elementary factors (Proposition 1);
    the sweep S_L^{-1} b (products of (I + E_d)) equals a dense triangular solve,
    and likewise for S_U."""
    w, A, dec, sw = _problem(23, 3, 3, medium="layered", seed=6)
    S = sw.dense_S()
    d = _diag_masks(dec)
    E = np.where(d[:, None] == d[None, :] + 1, S, 0)     # blocks from diagonal d-1 into d
    F = np.where(d[:, None] == d[None, :] - 1, S, 0)
    assert np.abs(np.where(d[:, None] == d[None, :], S, 0)).max() == 0.0   # no diagonal blocks
    assert np.allclose(E + F, S, atol=0, rtol=0)
    I = np.eye(len(d))
    SL, SU = I - E, I - F
    prod = I.copy()
    for dd in range(3, dec.Ng + 2):
        Ed = np.where((d[:, None] == dd) & (d[None, :] == dd - 1), S, 0)
        prod = prod @ (I - Ed)
    assert np.abs(prod - SL).max() < 1e-13
    b = dec.unflatten(W.random_complex(len(d), 7))
    bf = dec.flatten(b)
    assert _rel(dec.flatten(sw.inv_SL(b)), np.linalg.solve(SL, bf)) < 1e-12
    assert _rel(dec.flatten(sw.inv_SU(b)), np.linalg.solve(SU, bf)) < 1e-12
    assert _rel(dec.flatten(sw.sgs(b)), np.linalg.solve(SU, np.linalg.solve(SL, bf))) < 1e-12


def test_block_jacobi_bands_against_dense():
    """Each band of B_L^{-1} equals the dense S_L^{-1} applied to the band-restricted
    right-hand side, read on the diagonals the band owns; the residual half-step
    uses rho = b - (I - S) x'."""
    w, A, dec, sw = _problem(22, 2, 4, medium="layered", seed=8)     # Ng = 5, N1 = 2: 2 bands each way
    S = sw.dense_S()
    d = _diag_masks(dec)
    I = np.eye(len(d))
    SL = I - np.where(d[:, None] == d[None, :] + 1, S, 0)
    SU = I - np.where(d[:, None] == d[None, :] - 1, S, 0)
    b = dec.unflatten(W.random_complex(len(d), 9))
    bf = dec.flatten(b)
    BL = bands(dec.N1, dec.Ng, "L")
    assert len(BL) >= 2
    xh = np.zeros_like(bf)
    for g, (lo, hi) in enumerate(BL):
        band = (d >= lo) & (d <= hi)
        own = (d > lo) & (d <= hi) | ((d == lo) if g == 0 else False)
        xh[own] = np.linalg.solve(SL, np.where(band, bf, 0))[own]
    assert _rel(dec.flatten(sw.block_jacobi_L(b)), xh) < 1e-12
    rho = bf - (I - S) @ xh
    y = np.zeros_like(bf)
    for g, (lo, hi) in enumerate(bands(dec.N1, dec.Ng, "U")):
        band = (d >= lo) & (d <= hi)
        own = (d >= lo) & (d < hi) | ((d == hi) if g == 0 else False)
        y[own] = np.linalg.solve(SU, np.where(band, rho, 0))[own]
    assert _rel(dec.flatten(sw.bsp(b)), xh + y) < 1e-12


@pytest.mark.parametrize("N1,N2", [(2, 4), (2, 6), (3, 5)])
def test_leading_band_is_an_exact_substitution(N1, N2):
    """Section 5 without the dense restatement: S_L is block lower triangular by
    diagonals, so S_L^{-1} b on the diagonals of the first forward band depends only on
    b there and on that band's own blocks.  For b supported on the first band (its
    shared last diagonal included), B_L^{-1} b must equal S_L^{-1} b (the product of
    Proposition 1's factors) on those diagonals; with b zero on the shared diagonal as
    well, the other bands start from zero and B_L^{-1} b vanishes beyond the band (no
    propagation between bands in one block Jacobi half-step).  The same for the first
    backward band (top-right corner) and S_U.  The literal additive sum counts the
    shared diagonal twice and fails the first check."""
    w, A, dec, sw = _problem(6 * max(N1, N2), N1, N2, medium="layered", seed=10 + N2)
    n = sum(dec.side_length(*ij) for ij in dec.slots)
    full = dec.unflatten(W.random_complex(n, 12))

    def on(diags):
        return {ij: (v.copy() if dec.diagonal(ij[0]) in diags else np.zeros_like(v)) for ij, v in full.items()}

    def vec(x, pred):
        return np.concatenate([x[ij] for ij in dec.slots if pred(dec.diagonal(ij[0]))])

    (lo, hi) = bands(dec.N1, dec.Ng, "L")[0]
    assert len(bands(dec.N1, dec.Ng, "L")) >= 2 and lo == 2
    b = on(set(range(lo, hi + 1)))
    assert _rel(vec(sw.block_jacobi_L(b), lambda d: d <= hi), vec(sw.inv_SL(b), lambda d: d <= hi)) < 1e-13
    b = on(set(range(lo, hi)))
    x, ex = sw.block_jacobi_L(b), sw.inv_SL(b)
    assert _rel(vec(x, lambda d: d <= hi), vec(ex, lambda d: d <= hi)) < 1e-13
    assert np.abs(vec(x, lambda d: d > hi)).max() == 0.0 and np.abs(vec(ex, lambda d: d > hi)).max() > 0.0

    (lo, hi) = bands(dec.N1, dec.Ng, "U")[0]
    assert hi == dec.Ng + 1
    r = on(set(range(lo, hi + 1)))
    assert _rel(vec(sw.block_jacobi_U(r), lambda d: d >= lo), vec(sw.inv_SU(r), lambda d: d >= lo)) < 1e-13
    r = on(set(range(lo + 1, hi + 1)))
    y, ey = sw.block_jacobi_U(r), sw.inv_SU(r)
    assert _rel(vec(y, lambda d: d >= lo), vec(ey, lambda d: d >= lo)) < 1e-13
    assert np.abs(vec(y, lambda d: d < lo)).max() == 0.0 and np.abs(vec(ey, lambda d: d < lo)).max() > 0.0


@pytest.mark.parametrize("N1,N2", [(2, 2), (4, 2), (3, 2), (2, 1)])
def test_bsp_with_one_band_equals_sgs(N1, N2):
    """One band (Ng - 1 <= N1): B_L = S_L and the two half-steps give exactly S_U^{-1} S_L^{-1}."""
    w, A, dec, sw = _problem(24, N1, N2, medium="layered", seed=1)
    assert len(bands(N1, dec.Ng, "L")) == 1
    r = W.random_complex(w.N, 2)
    assert _rel(sw.precondition(r, "BSP"), sw.precondition(r, "SP")) < 1e-13


def test_preconditioner_is_linear():
    w, A, dec, sw = _problem(26, 3, 3, medium="layered", seed=3)
    r1, r2 = W.random_complex(w.N, 4), W.random_complex(w.N, 5)
    a = 0.7 - 1.3j
    for kind in ("SP", "BSP"):
        lhs = sw.precondition(a * r1 + r2, kind)
        rhs = a * sw.precondition(r1, kind) + sw.precondition(r2, kind)
        assert _rel(lhs, rhs) < 1e-13


# ------------------------------------------------------------------- Krylov
def test_fgmres_solves_dense_system():
    rng = np.random.default_rng(0)
    n = 60
    M = np.eye(n) * 4 + (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * 0.2
    b = rng.normal(size=n) + 0j
    x, it, rr = fgmres(lambda v: M @ v, lambda v: v, b, tol=1e-12, restart=10)
    assert rr < 1e-12 and _rel(x, np.linalg.solve(M, b)) < 1e-10
    assert it > 10      # restarted at least once


@pytest.mark.parametrize("kind", ["SP", "BSP"])
def test_fgmres_with_sweeps_matches_direct_solve(kind):
    w, A, dec, sw = _problem(40, 3, 2, medium="layered", seed=7, xcuts=[0, 14, 27, 40])
    b = w.h ** 2 * w.f[0]
    x, it, rr = fgmres(lambda v: A @ v, lambda v: sw.precondition(v, kind), b, tol=1e-12)
    assert rr <= 1e-12
    assert _rel(x, spla.spsolve(A.tocsc(), b)) < 1e-9


# ------------------------------------------------------------------ adjoint
def _adjoint_case():
    n, h = 31, 1.0 / 32
    w = W.workload("custom", n=n, N1=2, N2=2, medium="layered", seed=3, nrhs=3, ppw=10)
    rec = np.arange((n - 1) * n + 1, n * n, 3)
    rng = np.random.default_rng(1)
    d = rng.normal(size=(3, len(rec))) * 1e-4 + 1j * rng.normal(size=(3, len(rec))) * 1e-4
    return w, rec, d


def test_gradient_matches_central_differences():
    w, rec, d = _adjoint_case()
    J, g, _ = misfit_gradient_direct(w.n, w.h, w.omega, w.m2, w.f, rec, d)
    rng = np.random.default_rng(2)
    for k in range(3):
        dm = W.smooth_random_field(w.n, 20 + k, 0.2, w.h).reshape(-1) * 1e-3 * w.m2.max()
        eps = 1.0
        Jp = misfit_value(w.n, w.h, w.omega, w.m2 + eps * dm, w.f, rec, d)
        Jm = misfit_value(w.n, w.h, w.omega, w.m2 - eps * dm, w.f, rec, d)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - g @ dm) <= 1e-4 * abs(fd)


def test_operator_derivative_matches_differences():
    w = W.workload("custom", n=9, N1=1, N2=1, medium="layered", seed=1)
    da = operator_diagonal_derivative(w.n, w.h, w.omega, w.m2)
    e = 1e-6 * w.m2
    Ap = assemble_operator(w.n, w.h, w.omega, w.m2 + e).diagonal()
    Am = assemble_operator(w.n, w.h, w.omega, w.m2 - e).diagonal()
    assert np.abs((Ap - Am) / (2 * e) - da).max() <= 1e-6 * np.abs(da).max()


def test_iterative_adjoint_matches_direct_adjoint():
    w, rec, d = _adjoint_case()
    J, g, U = misfit_gradient_direct(w.n, w.h, w.omega, w.m2, w.f, rec, d)
    A = assemble_operator(w.n, w.h, w.omega, w.m2)
    dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    sw = Sweeper(dec)
    solve = lambda rhs: fgmres(lambda v: A @ v, lambda v: sw.precondition(v, "BSP"), rhs, tol=1e-13)[0]
    J2, g2, U2 = misfit_gradient_iterative(w.n, w.h, w.omega, w.m2, w.f, rec, d, solve)
    assert abs(J2 - J) <= 1e-8 * J
    assert _rel(g2, g) < 1e-8
