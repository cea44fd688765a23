"""Seeded synthetic inputs for the Helmholtz workloads.

This module is the only code shared by the CPU oracle (``oracle/``) and the
GPU library (``paper_2209_10886_gb300``).  It produces *inputs* only — grids,
partitions, squared-slowness fields, sources, receivers — and contains none of
the method's arithmetic (no stencil, no transmission operator, no sweep, no
Krylov step).

Conventions
-----------
* The grid has ``n x n`` interior nodes ``x_{a,b} = (a h, b h)`` with
  ``a, b = 1..n`` and ``h = 1/(n+1)``.  Arrays are stored row-major with the
  y index ``b`` slowest: flat index ``p = (b-1)*n + (a-1)``.
* ``m2`` is the squared slowness ``1/c(x)^2``; the wavenumber is
  ``kappa = omega * sqrt(m2)``.
* A checkerboard partition is given by node offsets ``xcuts`` (length N1+1)
  and ``ycuts`` (length N2+1); column ``i1`` of subdomains owns x-nodes
  ``xcuts[i1-1] .. xcuts[i1]-1`` (0-based), row ``i2`` likewise in y.

The synthetic workloads stand in for the paper's finite-element scattering
benchmark (Section 6 of the paper), which cannot be regenerated here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "even_cuts",
    "layered_random_medium",
    "smooth_random_field",
    "gaussian_source",
    "workload",
    "WORKLOADS",
]


def even_cuts(n: int, parts: int, block: int | None = None) -> np.ndarray:
    """Node offsets splitting ``n`` nodes into ``parts`` pieces.

    With ``block`` given, every piece but the last has ``block`` nodes and the
    last takes the remainder (e.g. 1023 = 7*128 + 127).  Without it the split
    is as even as possible, larger pieces first.
    """
    if block is not None:
        sizes = [block] * (parts - 1) + [n - block * (parts - 1)]
    else:
        q, r = divmod(n, parts)
        sizes = [q + 1] * r + [q] * (parts - r)
    if min(sizes) < 1:
        raise ValueError("empty subdomain in partition")
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def smooth_random_field(n: int, seed: int, corr_len: float, h: float) -> np.ndarray:
    """Seeded standard-normal field smoothed by a Gaussian of width ``corr_len``.

    The white noise comes from NumPy's PCG64 generator.  Smoothing is a
    Gaussian filter of standard deviation ``corr_len / h`` grid cells applied
    in Fourier space to the mirror-extended field (reflecting boundaries).
    The result is scaled so that ``max|delta| = 1``.  Shape ``(n, n)``,
    indexed ``[b, a]`` (y slowest).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n))
    sig = corr_len / h
    ext = np.concatenate([w, w[::-1, :]], axis=0)
    ext = np.concatenate([ext, ext[:, ::-1]], axis=1)
    ky = np.fft.fftfreq(2 * n)[:, None]
    kx = np.fft.rfftfreq(2 * n)[None, :]
    filt = np.exp(-2.0 * (math.pi * sig) ** 2 * (kx * kx + ky * ky))
    sm = np.fft.irfft2(np.fft.rfft2(ext) * filt, s=ext.shape)[:n, :n]
    sm -= sm.mean()
    return sm / np.abs(sm).max()


def layered_random_medium(n: int, seed: int, h: float) -> np.ndarray:
    """Wave speed ``c(x)`` (km/s) of the three-layer medium with a +-10% perturbation.

    Depth is ``z = 1 - y``.  ``c = 1.5`` for ``z < 1/3``, ``2.5`` for
    ``1/3 <= z < 2/3`` and ``3.5`` below; then ``c <- c (1 + 0.1 delta)`` with
    ``delta`` from :func:`smooth_random_field` (correlation length 0.05).
    Shape ``(n, n)`` indexed ``[b, a]``.
    """
    y = (np.arange(1, n + 1) * h)[:, None]
    z = 1.0 - y
    c = np.where(z < 1.0 / 3.0, 1.5, np.where(z < 2.0 / 3.0, 2.5, 3.5))
    c = np.broadcast_to(c, (n, n)).astype(np.float64)
    delta = smooth_random_field(n, seed, 0.05, h)
    return c * (1.0 + 0.1 * delta)


def gaussian_source(n: int, h: float, centre, sigma: float) -> np.ndarray:
    """Normalised 2-D Gaussian ``exp(-|x-x_s|^2/(2 s^2)) / (2 pi s^2)`` on the grid.

    Returns a complex128 vector of length ``n*n`` (y slowest).
    """
    xs = np.arange(1, n + 1) * h
    gx = np.exp(-((xs - centre[0]) ** 2) / (2 * sigma * sigma))
    gy = np.exp(-((xs - centre[1]) ** 2) / (2 * sigma * sigma))
    f = np.outer(gy, gx) / (2 * math.pi * sigma * sigma)
    return f.reshape(-1).astype(np.complex128)


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, medium, partition, right-hand sides."""

    name: str
    n: int
    N1: int
    N2: int
    xcuts: np.ndarray
    ycuts: np.ndarray
    omega: float
    m2: np.ndarray            # (n*n,) float64, y slowest
    f: np.ndarray             # (nrhs, n*n) complex128
    rec_idx: np.ndarray | None = None   # (nrec,) int64 flat node indices
    m2_true: np.ndarray | None = None   # for the misfit workload
    description: str = ""

    @property
    def h(self) -> float:
        return 1.0 / (self.n + 1)

    @property
    def N(self) -> int:
        return self.n * self.n

    @property
    def nrhs(self) -> int:
        return self.f.shape[0]


def _omega_for_ppw(c_min: float, h: float, ppw: float) -> float:
    # smallest wavelength 2*pi*c_min/omega equals ppw grid cells
    return 2.0 * math.pi * c_min / (ppw * h)


def _line_sources(n, h, count, depth):
    y = 1.0 - depth
    return np.stack([gaussian_source(n, h, ((s + 0.5) / count, y), 2 * h) for s in range(count)])


def workload(name: str, **over) -> Workload:
    """Build one of the named workloads (``tiny``, ``plain_mixed``, ``batching``,
    ``differentiation``, ``large``) or a small custom one (``custom``).

    ``custom`` keyword arguments: ``n, N1, N2, ppw, medium ('const'|'layered'),
    seed, nrhs, xcuts, ycuts``.
    """
    if name == "tiny":
        # 127x127, 2x2 (64/63), constant kappa at 10 points per wavelength
        n = 127
        h = 1.0 / (n + 1)
        cuts = np.array([0, 64, 127])
        m2 = np.ones(n * n)
        omega = 2 * math.pi / (10 * h)
        f = gaussian_source(n, h, (0.3, 0.4), 2 * h)[None, :]
        return Workload(name, n, 2, 2, cuts, cuts.copy(), omega, m2, f,
                        description="127^2, 2x2, constant kappa 10 ppw, 1 Gaussian source")
    if name == "plain_mixed":
        n = 1023
        h = 1.0 / (n + 1)
        cuts = even_cuts(n, 8, 128)
        c = layered_random_medium(n, 0, h)
        omega = _omega_for_ppw(c.min(), h, 8.0)
        nrhs = over.get("nrhs", 1)
        # one point source, or (nrhs > 1) a line of sources at depth 0.05 as in the batching workload
        f = gaussian_source(n, h, (0.3, 0.4), 2 * h)[None, :] if nrhs == 1 else _line_sources(n, h, nrhs, 0.05)
        return Workload(name, n, 8, 8, cuts, cuts.copy(), omega, (1.0 / c**2).reshape(-1), f,
                        description=f"1023^2, 8x8, layered+random medium 8 ppw, {nrhs} source(s)")
    if name == "batching":
        n = 1535
        h = 1.0 / (n + 1)
        sizes = [128, 127, 129, 127, 130, 127, 131, 127, 127, 128, 127, 127]
        cuts = np.concatenate([[0], np.cumsum(sizes)])
        c = layered_random_medium(n, 0, h)
        omega = _omega_for_ppw(c.min(), h, 8.0)
        nrhs = over.get("nrhs", 64)
        f = _line_sources(n, h, 64, 0.05)[:nrhs]
        return Workload(name, n, 12, 12, cuts, cuts.copy(), omega, (1.0 / c**2).reshape(-1), f,
                        description="1535^2, 12x12 uneven, layered+random 8 ppw, 64 sources")
    if name == "differentiation":
        n = 511
        h = 1.0 / (n + 1)
        cuts = even_cuts(n, 4, 128)
        delta = smooth_random_field(n, 1, 0.05, h)
        c = 2.5 * (1.0 + 0.1 * delta)
        m2 = (1.0 / c**2).reshape(-1)
        omega = _omega_for_ppw(c.min(), h, 8.0)
        xs = np.arange(1, n + 1) * h
        bump = np.exp(-(((xs[None, :] - 0.5) ** 2 + (xs[:, None] - 0.5) ** 2) / (2 * 0.1**2)))
        m2_true = m2 * (1.0 + 0.05 * bump.reshape(-1))
        top = n  # b = n (1-based), the top row
        f = np.stack([gaussian_source(n, h, ((32 * s + 16) * h, top * h), 2 * h) for s in range(16)])
        rec = np.array([(top - 1) * n + (4 * r + 2 - 1) for r in range(128)], dtype=np.int64)
        return Workload(name, n, 4, 4, cuts, cuts.copy(), omega, m2, f, rec_idx=rec, m2_true=m2_true,
                        description="511^2, 4x4, smooth medium, 16 sources, 128 receivers")
    if name == "large":
        n = 4095
        h = 1.0 / (n + 1)
        cuts = even_cuts(n, 16, 256)
        c = layered_random_medium(n, 0, h)
        omega = _omega_for_ppw(c.min(), h, 10.0)
        nrhs = over.get("nrhs", 32)
        f = _line_sources(n, h, 32, 0.05)[:nrhs]
        return Workload(name, n, 16, 16, cuts, cuts.copy(), omega, (1.0 / c**2).reshape(-1), f,
                        description="4095^2, 16x16, layered+random 10 ppw, 32 sources")
    if name == "custom":
        n = over["n"]
        h = 1.0 / (n + 1)
        N1, N2 = over.get("N1", 2), over.get("N2", 2)
        xcuts = np.asarray(over["xcuts"]) if "xcuts" in over else even_cuts(n, N1)
        ycuts = np.asarray(over["ycuts"]) if "ycuts" in over else even_cuts(n, N2)
        ppw = over.get("ppw", 10.0)
        nrhs = over.get("nrhs", 1)
        if over.get("medium", "const") == "const":
            c = np.ones((n, n))
        else:
            c = layered_random_medium(n, over.get("seed", 0), h)
        omega = _omega_for_ppw(c.min(), h, ppw)
        rng = np.random.Generator(np.random.PCG64(over.get("seed", 0) + 1000))
        centres = [(0.3, 0.4)] + [tuple(rng.uniform(0.15, 0.85, 2)) for _ in range(nrhs - 1)]
        f = np.stack([gaussian_source(n, h, cc, 2 * h) for cc in centres])
        return Workload("custom", n, N1, N2, xcuts, ycuts, omega, (1.0 / c**2).reshape(-1), f,
                        description=f"{n}^2, {N1}x{N2}, custom")
    raise KeyError(name)


WORKLOADS = ("tiny", "plain_mixed", "batching", "differentiation", "large")


def random_complex(shape, seed: int) -> np.ndarray:
    """Seeded complex128 array with standard-normal real and imaginary parts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
