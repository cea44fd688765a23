"""Pade-type high-order absorbing transmission operator (finite-difference form).

TEST INFRASTRUCTURE ONLY, like the rest of :mod:`oracle`.

The paper transmits between subdomains with a Pade-type HABC with
``N_pade = 8`` auxiliary fields and rotation ``phi = pi/3`` (Section 6,
experimental setup; Section 3 names the HABCs of its references as the
transmission conditions).  It gives no formula; the operator is the rotated
Pade approximation of the square-root (one-way) operator of the published
HABCs it cites:

    d_n u = i k sqrt(1 + Delta_G / k^2) u,
    sqrt(1 + z) ~ e^{i phi / 2} R_N((1 + z) e^{-i phi} - 1),
    R_N(w) = 1 + sum_{l=1..N} a_l w / (1 + b_l w),
    a_l = 2/M sin^2(l pi / M),  b_l = cos^2(l pi / M),  M = 2N + 1,

R_N being the [N/N] Pade approximant of sqrt(1 + w) at w = 0, and the
rotation moving its branch cut off the negative real axis so that evanescent
modes (z < -1) are damped.  The auxiliary-field form of the references
(phi_l = w / (1 + b_l w) u on the boundary) is the same operator; here each
interface side carries it as the dense matrix it defines on the side's points.

Readings taken where the paper is silent: Delta_G is the 3-point second difference
along the side with spacing h and homogeneous Neumann ends (no corner
treatment: the fields of one side do not see the other sides); k is the edge
wavenumber kappa_e of each point; the HABC acts on interfaces only, the outer
boundary keeps the first-order condition of the global problem, so the DD
fixed point is the global discrete solution.
"""
import numpy as np


def pade_coefficients(N):
    """``(a_l, b_l)``, l = 1..N, of the [N/N] Pade approximant of sqrt(1 + w)."""
    M = 2 * N + 1
    theta = np.arange(1, N + 1) * np.pi / M
    return 2.0 / M * np.sin(theta) ** 2, np.cos(theta) ** 2


def pade_sqrt(w, N):
    """``R_N(w) = 1 + sum_l a_l w / (1 + b_l w)`` (scalar or array ``w``)."""
    a, b = pade_coefficients(N)
    w = np.asarray(w, dtype=np.complex128)
    out = np.ones_like(w)
    for al, bl in zip(a, b):
        out = out + al * w / (1.0 + bl * w)
    return out


def rotated_sqrt(z, N, phi):
    """``e^{i phi/2} R_N((1 + z) e^{-i phi} - 1)``, the rotated Pade square root."""
    z = np.asarray(z, dtype=np.complex128)
    return np.exp(0.5j * phi) * pade_sqrt((1.0 + z) * np.exp(-1j * phi) - 1.0, N)


def tangential_laplacian(L, h):
    """3-point second difference on L points with spacing h, Neumann ends."""
    D = np.zeros((L, L))
    idx = np.arange(L)
    D[idx, idx] = -2.0
    D[idx[:-1], idx[:-1] + 1] = 1.0
    D[idx[1:], idx[1:] - 1] = 1.0
    if L >= 1:
        D[0, 0] += 1.0          # ghost phi_0 = phi_1
        D[-1, -1] += 1.0        # ghost phi_{L+1} = phi_L
    return D / h ** 2


def side_operator(kappa, h, N, phi):
    """The matrix ``T = i diag(k) e^{i phi/2} R_N(W)``, ``W = (I + Z) e^{-i phi} - I``,
    ``Z = diag(1/k^2) Delta_G``, on the L points of one side (``kappa``: their k)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    L = kappa.size
    Id = np.eye(L, dtype=np.complex128)
    Z = (1.0 / kappa ** 2)[:, None] * tangential_laplacian(L, h)
    W = (Id + Z) * np.exp(-1j * phi) - Id
    a, b = pade_coefficients(N)
    R = Id.copy()
    for al, bl in zip(a, b):
        R = R + al * np.linalg.solve((Id + bl * W).T, W.T).T      # a_l W (I + b_l W)^{-1}
    return 1j * kappa[:, None] * np.exp(0.5j * phi) * R
