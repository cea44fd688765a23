"""Pins of the oracle's Pade-type HABC transmission (oracle/habc.py): the operator
the paper transmits with (Sections 3 and 6: N_pade = 8, phi = pi/3), in the
finite-difference form of this build.

* R_N is the [N/N] Pade approximant of sqrt(1 + w): it agrees with the square
  root to O(w^(2N+1)) (the Taylor series), a check that a wrong coefficient fails.
* The rotation of the branch cut gives the right branch for evanescent modes
  (z < -1: sqrt(1+z) = i sqrt(-1-z), the decaying one) and converges with N;
  without it the evanescent values are wrong.
* The side matrix acts on the Neumann cosine modes of the side as the scalar
  symbol at the discrete eigenvalue (exact, constant k).
* N = 0 without rotation is the impedance condition T = i kappa_e.
* With the HABC on every interface, the exact interface solve reproduces the
  global discrete solution (the DD fixed point), and the BSP-preconditioned
  interface GMRES needs fewer iterations than with the Robin condition.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import Decomposition, Sweeper, assemble_operator, habc
from oracle.krylov import fgmres


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("N", [1, 2, 3])
def test_pade_approximant_agrees_with_the_taylor_series(N):
    """R_N - sqrt(1 + w) = O(w^(2N+1)): halving w divides the error by 2^(2N+1)."""
    for w in (0.1, -0.1, 0.1j):
        e1 = abs(habc.pade_sqrt(w, N) - np.sqrt(1 + w))
        e2 = abs(habc.pade_sqrt(w / 2, N) - np.sqrt(1 + w / 2))
        assert e1 < 0.05 * abs(w) ** (2 * N + 1)
        assert 0.7 < (e1 / e2) / 2 ** (2 * N + 1) < 1.3, (w, e1, e2)


def test_rotated_branch_is_the_decaying_one_and_converges():
    zp = np.linspace(-0.9, 0.5, 50)               # propagating (and above)
    ze = np.linspace(-6.0, -1.2, 50)              # evanescent
    exact_p, exact_e = np.sqrt(1 + zp + 0j), 1j * np.sqrt(-1 - ze)
    e8 = max(np.abs(habc.rotated_sqrt(zp, 8, np.pi / 3) - exact_p).max(),
             np.abs(habc.rotated_sqrt(ze, 8, np.pi / 3) - exact_e).max())
    e16 = max(np.abs(habc.rotated_sqrt(zp, 16, np.pi / 3) - exact_p).max(),
              np.abs(habc.rotated_sqrt(ze, 16, np.pi / 3) - exact_e).max())
    assert e8 < 1e-2 and e16 < 1e-4 and e16 < e8 / 100
    assert np.abs(habc.rotated_sqrt(ze, 8, 0.0) - exact_e).max() > 1.0    # no rotation: wrong


def test_side_matrix_on_neumann_modes_is_the_symbol():
    L, h, kappa, N, phi = 37, 0.01, 55.0, 8, np.pi / 3
    T = habc.side_operator(np.full(L, kappa), h, N, phi)
    j = np.arange(L)
    for k in (0, 1, 5, 17, 36):
        v = np.cos(np.pi * k * (j + 0.5) / L)
        lam = -(2.0 - 2.0 * np.cos(np.pi * k / L)) / h ** 2
        sym = 1j * kappa * habc.rotated_sqrt(lam / kappa ** 2, N, phi)
        assert rel(T @ v, sym * v) < 1e-10, k


CASE = dict(n=60, N1=3, N2=2, medium="layered", seed=3, xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60])


def test_zeroth_order_unrotated_habc_is_the_impedance_condition():
    w = W.workload("custom", **CASE)
    r = W.random_complex((1, w.N), 5)[0]
    a = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission="habc", n_pade=0, phi=0.0))
    b = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission="impedance"))
    for kind in ("BSP", "SP"):
        assert rel(a.precondition(r, kind), b.precondition(r, kind)) < 1e-13


def test_habc_decomposition_fixed_point_is_the_global_solution():
    w = W.workload("custom", **CASE)
    A = assemble_operator(w.n, w.h, w.omega, w.m2).tocsc()
    r = W.random_complex((1, w.N), 5)[0]
    sw = Sweeper(Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission="habc"))
    assert rel(sw.precondition(r, "exact"), spla.spsolve(A, r)) < 1e-12


def test_habc_needs_fewer_interface_iterations_than_robin():
    w = W.workload("custom", n=119, N1=5, N2=3, medium="layered", seed=3)
    r = w.h ** 2 * w.f[0]
    its = {}
    for tr in ("optimized", "habc"):
        dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, transmission=tr, tc_scale=0.5)
        sw = Sweeper(dec)
        b = dec.flatten(sw.lifting_traces(r))
        _, its[tr], rr = fgmres(lambda v: v - dec.flatten(sw.apply_S(dec.unflatten(v))),
                                lambda v: dec.flatten(sw.bsp(dec.unflatten(v))), b, tol=1e-6, restart=100, maxit=300)
        assert rr <= 1e-6
    print("BSP interface GMRES iterations:", its)
    assert its["habc"] < its["optimized"]


def test_habc_local_problem_is_a_boundary_modification_of_the_robin_one():
    """The HABC local matrix differs from a Robin one only by the side blocks on the
    boundary points, A_habc = A_robin - P C P^T, so its boundary block follows from
    the Robin one in the boundary space: K_habc = (I - K_robin C)^{-1} K_robin (the
    push-through form of the Woodbury identity; P may repeat a corner node)."""
    import oracle.decomposition as odec
    w = W.workload("custom", **CASE)
    args = (w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    dh = Decomposition(*args, transmission="habc")
    db = Decomposition(*args, transmission="optimized", tc_scale=0.5)
    i = max(dh.subdomains, key=lambda s: len(dh.neighbours(s)))       # the most interface sides
    sides = list(dh.neighbours(i))
    pts = np.concatenate([dh._edges[(i, j)][0] for j in sides])        # boundary points, side by side
    Mi = dh.local_matrix(i).shape[0]
    P = np.zeros((Mi, pts.size))
    P[pts, np.arange(pts.size)] = 1.0
    C = np.zeros((pts.size, pts.size), dtype=np.complex128)
    o = 0
    for j in sides:
        L = len(dh._edges[(i, j)][0])
        Ch = odec.ghost_matrix(dh._edges[(i, j)][1])
        Cb = np.diag(odec.ghost_factor(db._edges[(i, j)][1]))
        C[o:o + L, o:o + L] = Ch - Cb
        o += L
    Ah, Ab = dh.local_matrix(i).toarray(), db.local_matrix(i).toarray()
    assert np.abs(Ah - (Ab - P @ C @ P.T)).max() < 1e-12
    Kh = P.T @ np.linalg.solve(Ah, P)
    Kb = P.T @ np.linalg.solve(Ab, P)
    assert rel(np.linalg.solve(np.eye(pts.size) - Kb @ C, Kb), Kh) < 1e-10
