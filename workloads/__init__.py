"""Seeded synthetic inputs for the Helmholtz solver: media c(x), sources f, solver settings.

This module holds no arithmetic of the solution method.  It only draws the wavespeed
model, the right-hand sides and the scalar settings of each workload, so that the CPU
oracle (``oracle/``) and the GPU library (``paper_1811_12378_gb300``) can be fed the
same inputs without sharing any code of the method.

Layout of every grid array: numpy shape ``(nz, ny, nx)`` in C order, i.e. the linear
index of interior point (i, j, k) is ``i + nx*(j + ny*k)`` (x fastest).  Interior point
(i, j, k) sits at ``((i+1)h, (j+1)h, (k+1)h)``; the zero Dirichlet ghosts are implicit.

The paper's own media (eight high-speed anomalies, §7.3, shown only as a figure) and the
SEG/EAGE salt model (§8, a dataset not available here) cannot be recreated; the
Gaussian-bump and layered media below stand in for them in shape and speed range.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    """One solver workload: grid, medium, sources and the settings of the method.

    omega is the angular frequency; ppw the points per wavelength at the slowest speed.
    layer_cells / sigma_max describe the absorbing sponge; J, t, eps the contour
    (§6.1, §6.2); restart / k_in / rtol the outer FGMRES(m), inner GMRES steps and the
    relative-residual target.  ``c`` has shape (nz, ny, nx); ``f`` has shape
    (nrhs, nz, ny, nx) complex128.
    """

    name: str
    nx: int
    ny: int
    nz: int
    h: float
    omega: float
    layer_cells: int
    sigma_max: float
    J: int
    t: float
    eps: float
    restart: int
    k_in: int
    rtol: float
    c: np.ndarray
    f: np.ndarray
    qmax: int = 5
    reduction: float = 5.0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nrhs(self) -> int:
        return int(self.f.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def coords(nx: int, ny: int, nz: int, h: float):
    """Physical coordinates of the interior points, each of shape (nz, ny, nx)."""
    x = (np.arange(nx) + 1.0) * h
    y = (np.arange(ny) + 1.0) * h
    z = (np.arange(nz) + 1.0) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def medium_constant(nx, ny, nz, c0=1.0):
    return np.full((nz, ny, nx), float(c0))


def medium_gaussian_bumps(seed, nx, ny, nz, h, nbumps=8, width=0.1, amp_hi=0.4,
                          c_lo=1.0, c_hi=2.0, amp_lo=0.0):
    """c = clip(1 + sum_k a_k exp(-|x-x_k|^2 / (2 width^2)), c_lo, c_hi).

    a_k ~ U[amp_lo, amp_hi], centres x_k ~ U[0, 1]^3 (unit cube), all drawn from PCG64(seed).
    """
    g = _rng(seed)
    amps = g.uniform(amp_lo, amp_hi, size=nbumps)
    ctrs = g.uniform(0.0, 1.0, size=(nbumps, 3))
    X, Y, Z = coords(nx, ny, nz, h)
    c = np.ones((nz, ny, nx))
    for a, (cx, cy, cz) in zip(amps, ctrs):
        r2 = (X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2
        c += a * np.exp(-r2 / (2.0 * width * width))
    return np.clip(c, c_lo, c_hi)


def medium_layered(seed, nx, ny, nz, nlayers=5, c_lo=1.5, c_hi=4.5):
    """nlayers equal-thickness horizontal layers along z, c per layer ~ U[c_lo, c_hi]."""
    g = _rng(seed)
    vals = g.uniform(c_lo, c_hi, size=nlayers)
    k = np.arange(nz)
    layer = np.minimum((k * nlayers) // nz, nlayers - 1)
    c = np.empty((nz, ny, nx))
    c[:] = vals[layer][:, None, None]
    return c


def source_point(nx, ny, nz, h, idx, amplitude=None):
    """Discrete delta at grid index idx = (i, j, k); default value 1/h^3."""
    f = np.zeros((nz, ny, nx), dtype=np.complex128)
    i, j, k = idx
    f[k, j, i] = (1.0 / h ** 3) if amplitude is None else amplitude
    return f


def source_gaussian(nx, ny, nz, h, centre, sigma):
    """f = exp(-|x - centre|^2 / (2 sigma^2)), peak 1."""
    X, Y, Z = coords(nx, ny, nz, h)
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    return np.exp(-r2 / (2.0 * sigma * sigma)).astype(np.complex128)


def random_core_index(g, nx, ny, nz, layer):
    """A grid index drawn uniformly from the points outside the absorbing layer."""
    lo = layer
    return (int(g.integers(lo, nx - lo)), int(g.integers(lo, ny - lo)),
            int(g.integers(lo, nz - lo)))


def random_field(seed, nvec, nx, ny, nz, dtype=np.complex128):
    """Standard complex normal vectors, shape (nvec, nz, ny, nx)."""
    g = _rng(seed)
    v = g.standard_normal((nvec, nz, ny, nx)) + 1j * g.standard_normal((nvec, nz, ny, nx))
    return v.astype(dtype)


def default_eps(nx, ny, nz):
    """Contour margin epsilon = min(1, 64/N): proportional to 1/omega at fixed ppw (§7.3)."""
    return min(1.0, 64.0 / max(nx, ny, nz))


def omega_for_ppw(c, h, ppw):
    """Angular frequency giving ppw points per wavelength at the slowest speed."""
    return 2.0 * math.pi * float(np.min(c)) / (ppw * h)


def point_source_32(seed: int = 0) -> Workload:
    """32^3 unit cube (h = 1/33), c = 1, 10 ppw, 8-cell sponge, centre point source, J = 4."""
    n = 32
    h = 1.0 / (n + 1)
    c = medium_constant(n, n, n)
    f = source_point(n, n, n, h, (n // 2, n // 2, n // 2))[None]
    return Workload("point_source_32", n, n, n, h, omega_for_ppw(c, h, 10.0), 8, 1.0,
                    4, 1.0, default_eps(n, n, n), 30, 4, 1e-8, c, f)


def gaussian_bumps_64(seed: int = 1) -> Workload:
    """64^3 (h = 1/65), c = 1 + 8 Gaussian bumps (width 0.1, amplitudes U[0,0.4]) clipped
    to [1, 2], 8 ppw at c_min, 8-cell sponge, one Gaussian source (sigma = 2h) at a seeded
    core point, J = 8 contour nodes."""
    n = 64
    h = 1.0 / (n + 1)
    c = medium_gaussian_bumps(seed, n, n, n, h)
    g = _rng(seed + 1000)
    i, j, k = random_core_index(g, n, n, n, 8)
    f = source_gaussian(n, n, n, h, ((i + 1) * h, (j + 1) * h, (k + 1) * h), 2.0 * h)[None]
    return Workload("gaussian_bumps_64", n, n, n, h, omega_for_ppw(c, h, 8.0), 8, 1.0,
                    8, 1.0, default_eps(n, n, n), 30, 4, 1e-8, c, f)


def gaussian_bumps(n: int, seed: int, ppw: float = 8.0, layer: int = 8, J: int = 8,
                   restart: int = 30) -> Workload:
    """The Gaussian-bump recipe of gaussian_bumps_64 at n^3 (h = 1/(n+1)): c = 1 + 8 bumps
    (width 0.1, amplitudes U[0,0.4]) clipped to [1, 2], ppw points per wavelength at c_min, one
    Gaussian source (sigma = 2h) at a seeded core point; media and sources for the learned
    preconditioner's training (64^3) and application (128^3, 192^3) sizes."""
    h = 1.0 / (n + 1)
    c = medium_gaussian_bumps(seed, n, n, n, h)
    g = _rng(seed + 1000)
    i, j, k = random_core_index(g, n, n, n, layer)
    f = source_gaussian(n, n, n, h, ((i + 1) * h, (j + 1) * h, (k + 1) * h), 2.0 * h)[None]
    return Workload(f"gaussian_bumps_{n}_{seed}", n, n, n, h, omega_for_ppw(c, h, ppw), layer,
                    1.0, J, 1.0, default_eps(n, n, n), restart, 4, 1e-8, c, f)


def spectral_bumps(n: int, seed: int, ppw: float = 2.25, layer: int = 8, J: int = 8,
                   restart: int = 30) -> Workload:
    """A Fourier spectral workload on the periodic n^3 box of spacing h = 1/n: background c = 1
    with 8 Gaussian bumps (width 0.1, amplitudes U[0.5, 1]) clipped to [1, 2], so the sampling
    rate is ppw points per wavelength in the background and up to twice that in the anomalies
    (the spectral runs sample 2.25 and 4.5), a layer-cell sponge at the box faces, one
    Gaussian source (sigma = 2h) at a seeded core point."""
    h = 1.0 / n
    c = medium_gaussian_bumps(seed, n, n, n, h, nbumps=8, width=0.1, amp_lo=0.5, amp_hi=1.0)
    g = _rng(seed + 1000)
    i, j, k = random_core_index(g, n, n, n, layer)
    f = source_gaussian(n, n, n, h, ((i + 1) * h, (j + 1) * h, (k + 1) * h), 2.0 * h)[None]
    return Workload(f"spectral_bumps_{n}_{seed}", n, n, n, h, omega_for_ppw(c, h, ppw), layer,
                    1.0, J, 1.0, default_eps(n, n, n), restart, 4, 1e-8, c, f)


def large_bumps_256(seed: int = 5, nsrc: int = 16):
    """256^3 (h = 1/257), c = 1 + 16 Gaussian bumps (width 0.1, amplitudes U[0, 2]) clipped to
    [1, 3], 8 ppw at c_min, 12-cell sponge, J = 8 contour nodes, FGMRES(40) with k_in = 4 to
    1e-8, nsrc unit point sources (value 1/h^3) at seeded core points.  The right-hand sides are
    returned as grid indices (nsrc fields of 256^3 complex128 values would be 4.3 GB on the
    host): (Workload with an empty f, [(i, j, k), ...])."""
    n = 256
    h = 1.0 / (n + 1)
    c = medium_gaussian_bumps(seed, n, n, n, h, nbumps=16, width=0.1, amp_hi=2.0, c_lo=1.0,
                              c_hi=3.0)
    g = _rng(seed + 1000)
    idx = [random_core_index(g, n, n, n, 12) for _ in range(nsrc)]
    f = np.zeros((0, 1, 1, 1), dtype=np.complex128)
    return (Workload("large_bumps_256", n, n, n, h, omega_for_ppw(c, h, 8.0), 12, 1.0, 8, 1.0,
                     default_eps(n, n, n), 40, 4, 1e-8, c, f), idx)


def small_case(seed: int, nx: int, ny: int, nz: int, nrhs: int = 1, ppw: float = 8.0,
               layer: int = 2, J: int = 4, restart: int = 10, k_in: int = 3,
               medium: str = "bumps") -> Workload:
    """A small ragged-shape workload for parity tests (any nx, ny, nz >= 1)."""
    h = 1.0 / (max(nx, ny, nz) + 1)
    if medium == "bumps":
        c = medium_gaussian_bumps(seed, nx, ny, nz, h, nbumps=4, width=0.2, amp_hi=0.8)
    elif medium == "layered":
        c = medium_layered(seed, nx, ny, nz, nlayers=3, c_lo=1.0, c_hi=2.0)
    else:
        c = medium_constant(nx, ny, nz)
    f = random_field(seed + 7, nrhs, nx, ny, nz)
    return Workload(f"small_{nx}x{ny}x{nz}", nx, ny, nz, h, omega_for_ppw(c, h, ppw), layer,
                    1.0, J, 1.0, 1.0, restart, k_in, 1e-8, c, f)


def layered_batch(seed: int = 3, sizes=(48, 64, 96), per_size: int = 4, nrhs: int = 4,
                  ppw: float = 8.0):
    """Instances of uneven grid sizes (per_size each of sizes), each with its own seeded
    layered medium (5 horizontal layers, c per layer ~ U[1.5, 4.5]), ppw points per
    wavelength at its c_min, an 8-cell sponge, J = 8 and nrhs unit point sources 1/h^3 at
    seeded core points."""
    out = []
    g = _rng(seed)
    idx = 0
    for N in sizes:
        for _ in range(per_size):
            h = 1.0 / (N + 1)
            c = medium_layered(seed * 1000 + idx, N, N, N, nlayers=5, c_lo=1.5, c_hi=4.5)
            f = np.zeros((nrhs, N, N, N), dtype=np.complex128)
            for r in range(nrhs):
                i, j, k = random_core_index(g, N, N, N, 8)
                f[r, k, j, i] = 1.0 / h ** 3
            out.append(Workload(f"layered_{N}_{idx}", N, N, N, h, omega_for_ppw(c, h, ppw), 8,
                                1.0, 8, 1.0, default_eps(N, N, N), 30, 4, 1e-8, c, f))
            idx += 1
    return out
