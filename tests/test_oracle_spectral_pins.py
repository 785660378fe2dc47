"""Pins of the oracle's Fourier spectral discretisation (§7.1 eq:eig-Laplacian-spectral), its
spectrum bound, and the regularised inverse-Laplacian inner preconditioner (§7.3), against
facts that do not come from the oracle: the paper's eigenvalue formula and radius bound, exact
derivatives of band-limited periodic functions, a DFT matrix built from its definition, and
dense linear algebra.  None of these needs a GPU.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import hz_oracle as O


def spectral_op(wl, kind="spectral"):
    return O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, kind=kind)


def laplacian_part(op, x):
    """(S x) alone: A x + m x + i a x = s S x."""
    return (op.apply(x) + op.m * x + 1j * op.a * x) / op.s


def plane_wave(nx, ny, nz, ix, iy, iz):
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    return (np.exp(2j * math.pi * iz * k / nz)[:, None, None]
            * np.exp(2j * math.pi * iy * j / ny)[None, :, None]
            * np.exp(2j * math.pi * ix * i / nx)[None, None, :])


def dft_matrix(n):
    """F[j, k] = exp(-2 pi i j k / n), element by element."""
    F = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        for k in range(n):
            F[j, k] = complex(math.cos(2 * math.pi * j * k / n), -math.sin(2 * math.pi * j * k / n))
    return F


@pytest.mark.parametrize("N", [6, 7, 8])
def test_plane_waves_have_the_papers_eigenvalues(N):
    """eq:eig-Laplacian-spectral: on an N^3 grid the normalised Laplacian s S has the plane
    wave of multi-index i as eigenvector with eigenvalue (l_min/N)^2 sum min(i_j^2, (N-i_j)^2),
    l_min = 2 pi c_min / (omega h) the sampling rate at the slowest speed."""
    wl = W.small_case(4, N, N, N, layer=1, ppw=3.0)
    op = spectral_op(wl)
    lmin = 2 * math.pi * float(wl.c.min()) / (wl.omega * wl.h)
    for (ix, iy, iz) in [(0, 0, 0), (1, 0, 0), (0, N - 1, 2), (N // 2, N // 2, N // 2),
                         (3, N - 2, 1)]:
        x = plane_wave(N, N, N, ix, iy, iz)
        lam = (lmin / N) ** 2 * sum(min(i * i, (N - i) ** 2) for i in (ix, iy, iz))
        assert np.allclose(op.s * laplacian_part(op, x), lam * x, rtol=1e-10,
                           atol=1e-10 * max(lam, 1.0))


def test_exact_derivatives_of_band_limited_functions():
    """-Delta of sin(2 pi x / Lx) cos(4 pi y / Ly) exp(2 pi i z / Lz) on the periodic box of
    lengths L = n h is (2pi/Lx)^2 + (4pi/Ly)^2 + (2pi/Lz)^2 times the function, exactly."""
    nx, ny, nz, h = 9, 8, 10, 0.07
    c = np.ones((nz, ny, nx))
    op = O.make_operator(c, h, 3.0, 0, 0.0, kind="spectral")
    Lx, Ly, Lz = nx * h, ny * h, nz * h
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    z = np.arange(nz) * h
    f = (np.exp(2j * math.pi * z / Lz)[:, None, None] * np.cos(4 * math.pi * y / Ly)[None, :, None]
         * np.sin(2 * math.pi * x / Lx)[None, None, :])
    k2 = (2 * math.pi / Lx) ** 2 + (4 * math.pi / Ly) ** 2 + (2 * math.pi / Lz) ** 2
    assert np.allclose(laplacian_part(op, f), k2 * f, rtol=1e-11, atol=1e-11 * k2)


def test_matches_a_dense_dft_construction():
    """S = F^H Lambda F / n with F the 3D DFT matrix (Kronecker product of 1D DFT matrices
    written from the definition) and Lambda from the wavenumbers min(i, n - i) 2 pi/(n h):
    the whole operator, mass and sponge included, against that dense matrix."""
    wl = W.small_case(9, 4, 3, 5, layer=1, ppw=3.0)
    op = spectral_op(wl)
    nx, ny, nz, h = op.nx, op.ny, op.nz, op.h
    F = np.kron(dft_matrix(nz), np.kron(dft_matrix(ny), dft_matrix(nx)))
    lam = np.zeros(op.n)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                lam[i + nx * (j + ny * k)] = sum(
                    (2 * math.pi * min(a, n - a) / (n * h)) ** 2
                    for a, n in ((i, nx), (j, ny), (k, nz)))
    S = F.conj().T @ np.diag(lam) @ F / op.n
    A = op.s * S - np.diag(op.m.ravel()) - 1j * np.diag(op.a.ravel())
    rng = np.random.Generator(np.random.PCG64(1))
    for _ in range(3):
        v = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
        z = 0.3 - 0.7j
        got = op.apply(v.reshape(op.shape), z).ravel()
        assert np.allclose(got, A @ v - z * v, rtol=1e-11, atol=1e-11 * np.abs(A).max())
    assert np.allclose(S, S.conj().T, atol=1e-9 * np.abs(S).max())  # Hermitian


@pytest.mark.parametrize("N", [6, 7])
def test_spectral_radius_bound(N):
    """§7.1: rho(s S) <= (3/4) l_min^2, with equality when N is even (the Nyquist mode
    N/2 along every axis); the spectrum box's b2 is s max(lambda) - min(m)."""
    wl = W.small_case(2, N, N, N, layer=1, ppw=2.25)
    op = spectral_op(wl)
    lmin = 2 * math.pi * float(wl.c.min()) / (wl.omega * wl.h)
    rho = op.s * O.spectral_eigenvalues(N, N, N, op.h).max()
    assert rho <= 0.75 * lmin ** 2 * (1 + 1e-12)
    if N % 2 == 0:
        assert rho == pytest.approx(0.75 * lmin ** 2, rel=1e-12)
    b1, b2, rho2 = O.spectrum_box(op)
    assert b2 == pytest.approx(rho - float(op.m.min()), rel=1e-12)
    assert b1 == pytest.approx(-float(op.m.max()), rel=1e-12)


@pytest.mark.parametrize("shape,layer", [((5, 4, 3), 1), ((4, 4, 4), 1)])
def test_spectrum_inside_box(shape, layer):
    """Lemma 3.1 for the spectral operator: every eigenvalue of the dense matrix (built column
    by column from unit vectors) lies in [b1, b2] x [-rho2, 0]."""
    wl = W.small_case(6, *shape, layer=layer, ppw=2.5)
    op = spectral_op(wl)
    A = np.column_stack([op.apply(e.reshape(op.shape)).ravel() for e in np.eye(op.n)])
    ev = np.linalg.eigvals(A)
    b1, b2, rho2 = O.spectrum_box(op)
    tol = 1e-9 * max(1.0, abs(b2))
    assert ev.real.min() >= b1 - tol and ev.real.max() <= b2 + tol
    assert ev.imag.min() >= -rho2 - tol and ev.imag.max() <= tol


def test_inverse_laplacian_on_plane_waves():
    """§7.3: the regularised inverse Laplacian has eigenvalues 1/max(lambda_i, 1) with lambda_i
    of eq:eig-Laplacian-spectral: it inverts s S on the modes above 1 and passes the ones
    below unchanged."""
    N = 8
    wl = W.small_case(3, N, N, N, layer=1, ppw=3.0)
    op = spectral_op(wl)
    P = O.invlap_preconditioner(op)
    lmin = 2 * math.pi * float(wl.c.min()) / (wl.omega * wl.h)
    seen = set()
    for (ix, iy, iz) in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (2, 1, 1), (4, 4, 4), (3, 7, 2)]:
        x = plane_wave(N, N, N, ix, iy, iz)
        lam = (lmin / N) ** 2 * sum(min(i * i, (N - i) ** 2) for i in (ix, iy, iz))
        seen.add(lam >= 1.0)
        assert np.allclose(P(x), x / max(lam, 1.0), rtol=1e-12, atol=1e-12)
        if lam >= 1.0:
            assert np.allclose(op.s * laplacian_part(op, P(x)), x, rtol=1e-10, atol=1e-10)
    assert seen == {True, False}  # both branches of the max are exercised


def test_spectral_fgmres_matches_dense_lu():
    """FGMRES with FCI on the spectral operator, with and without the inverse-Laplacian inner
    preconditioner, reaches 1e-8 and agrees with the dense solve within kappa * 1e-8; the
    contour is an ellipse of ratio t = 0.6 (§6.1)."""
    wl = W.small_case(12, 6, 5, 6, layer=1, ppw=2.5)
    op = spectral_op(wl)
    (_, _, _), nodes = O.setup_nodes(op, 6, 0.6, 1.0)
    A = np.column_stack([op.apply(e.reshape(op.shape)).ravel() for e in np.eye(op.n)])
    f = wl.f[0]
    u = np.linalg.solve(A, f.ravel())
    kappa = np.linalg.cond(A)
    for pre in (None, O.invlap_preconditioner(op)):
        res = O.solve(op, f, nodes, m=10, k_in=3, rtol=1e-8, max_cycles=40, inner_precond=pre)
        assert res.converged and res.rel_res_true <= 1e-8
        err = np.linalg.norm(res.u.ravel() - u) / np.linalg.norm(u)
        assert err <= kappa * 1e-8
