"""Oracle: a plain, slow complex128 CPU statement of the contour-integral Helmholtz solver.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference arm may import or call this module.  It shares no code with the
GPU library and imports nothing from it; both sides are fed the same seeded inputs by
``workloads``.

Everything is complex128 / float64 numpy, written step by step in the paper's order:

* operator      A = s*L_h - diag(m) - i*diag(a)            (§7.1 eq:stiff-mass, Case One;
                7-point or Fourier spectral L_h, eq:eig-Laplacian-spectral)
* bounds        rectangle B = [b1, b2] x [-rho2, 0]          (§3 Lemma 3.1)
* contour       nodes z_j and weights sigma_j                (§6.1, §6.2 eq:quad-points)
* poly params   z0, delta, q, nu, sweeps                     (§4.2 eq:fix-pt-conv)
* poly solve    fixed-point scheme                           (§4.2 eq:fix-pt-exp)
* FCI           quadrature, step d, inner GMRES              (§2 Algorithm 1)
* FGMRES        flexible GMRES with FCI as right precond.    (§2, after Algorithm 1)
* inner precond ILU(0) of the 7-point Laplacian, regularised inverse spectral
                Laplacian 1/max(lambda, 1)                   (§6.3, §7.3)
* Case Two      iC - I on (iu; u), its spectrum rectangle    (§3 eq:mat-2x2, Theorem
                and Algorithm 1 / FGMRES on it                thm:spectrum-2x2 and Remark)

Readings of points the paper leaves open (sign of the damping, normalisation, sponge
profile, delta search, stopping by a fixed sweep count, CGS2, Givens) are stated at each
function.  Every function here is pinned by a ``-m "not gpu"`` test against closed forms,
printed tables, brute force or dense linear algebra.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# ---------------------------------------------------------------------------------------
# Operator (§7.1, eq:stiff-mass; Case One of §3)
# ---------------------------------------------------------------------------------------

def sponge_depth(nx: int, ny: int, nz: int, layer: int) -> np.ndarray:
    """Depth into the absorbing layer in cells, shape (nz, ny, nx).

    Along one axis with n points, index i has edge distance e = min(i, n-1-i) and depth
    max(0, layer - e): ``layer`` at the outermost interior cell, 0 in the core.  The depth
    of a point is the largest over the three axes.
    """
    def axis(n):
        i = np.arange(n)
        e = np.minimum(i, n - 1 - i)
        return np.maximum(0, layer - e).astype(np.float64)
    dx, dy, dz = axis(nx), axis(ny), axis(nz)
    return np.maximum(np.maximum(dz[:, None, None], dy[None, :, None]), dx[None, None, :])


@dataclass
class Operator:
    """The normalised discrete Helmholtz operator A = s*L_h - diag(m) - i*diag(a).

    Reading of §7.1: the paper writes A = S - M + iD with S the negative discrete
    Laplacian scaled so that M_ii = l_min^2 / l_i^2 <= 1.  That is the physical operator
    -Delta_h - omega^2/c^2 times s = c_min^2/omega^2.  Case One (§3) needs the
    skew-Hermitian part to be -i times a PSD matrix, so the damping enters as -i*diag(a)
    and the spectrum lies in Im <= 0, which is what eq:quad-points assumes.  The damping
    is a quadratic sponge a = sigma_max * (depth/layer)^2 * m (positive in the layer,
    zero in the core, as §7.1 describes).  The physical system -Delta u - omega^2/c^2 u
    = f becomes A u = s f.
    """
    nx: int
    ny: int
    nz: int
    h: float
    s: float
    m: np.ndarray   # (nz, ny, nx) float64
    a: np.ndarray   # (nz, ny, nx) float64
    kind: str = "fd"  # "fd": 7-point, zero Dirichlet ghosts; "spectral": Fourier, periodic

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def apply(self, x: np.ndarray, z: complex = 0.0) -> np.ndarray:
        """(A - z I) x for one field x of shape (nz, ny, nx); zero Dirichlet ghosts (7-point)
        or the periodic Fourier spectral Laplacian (§7.1, S = F^H Lambda F)."""
        x = np.asarray(x, dtype=np.complex128).reshape(self.shape)
        if self.kind == "spectral":
            lam = spectral_eigenvalues(self.nx, self.ny, self.nz, self.h)
            lap = np.fft.ifftn(lam * np.fft.fftn(x))
            return self.s * lap - self.m * x - 1j * self.a * x - z * x
        xp = np.pad(x, 1)
        nb = (xp[1:-1, 1:-1, 2:] + xp[1:-1, 1:-1, :-2]
              + xp[1:-1, 2:, 1:-1] + xp[1:-1, :-2, 1:-1]
              + xp[2:, 1:-1, 1:-1] + xp[:-2, 1:-1, 1:-1])
        lap = (6.0 * x - nb) / (self.h * self.h)
        return self.s * lap - self.m * x - 1j * self.a * x - z * x


def spectral_eigenvalues(nx: int, ny: int, nz: int, h: float) -> np.ndarray:
    """Eigenvalues of -Delta under the Fourier spectral discretisation of the periodic box of
    nx x ny x nz points with spacing h, shape (nz, ny, nx), in the order of numpy's FFT.

    The mode with zero-based index i_d along an axis of n points is the plane wave
    exp(2 pi i i_d x / (n h)), sampled; its wavenumber is taken as 2 pi min(i_d, n - i_d)/(n h),
    the alias of smallest magnitude (§7.1 eq:eig-Laplacian-spectral uses min(i_d^2, (n-i_d)^2)).
    -Delta has the sum over the axes of the squared wavenumbers.  Times s = c_min^2/omega^2
    these are the paper's normalised (l_min/N)^2 sum min(i_d^2, (N - i_d)^2), since the
    sampling rate at c_min is l_min = 2 pi c_min / (omega h)."""
    def axis(n):
        i = np.arange(n)
        return (2.0 * math.pi * np.minimum(i, n - i) / (n * h)) ** 2
    ex, ey, ez = axis(nx), axis(ny), axis(nz)
    return ez[:, None, None] + ey[None, :, None] + ex[None, None, :]


def make_operator(c: np.ndarray, h: float, omega: float, layer: int,
                  sigma_max: float, kind: str = "fd") -> Operator:
    """Coefficients from the wavespeed c (shape (nz, ny, nx)): s, m = c_min^2/c^2, sponge a.
    kind "spectral" takes the Fourier spectral Laplacian on the periodic box (§7.1) with the
    same mass and sponge."""
    c = np.asarray(c, dtype=np.float64)
    nz, ny, nx = c.shape
    c_min = float(c.min())
    s = c_min * c_min / (omega * omega)
    m = (c_min * c_min) / (c * c)
    if layer > 0:
        d = sponge_depth(nx, ny, nz, layer)
        a = sigma_max * (d / layer) ** 2 * m
    else:
        a = np.zeros_like(m)
    if kind not in ("fd", "spectral"):
        raise ValueError(kind)
    return Operator(nx, ny, nz, float(h), s, m, a, kind)


# ---------------------------------------------------------------------------------------
# Spectrum rectangle (§3 Lemma 3.1) and contour (§6.1, §6.2)
# ---------------------------------------------------------------------------------------

def laplacian_extremes(nx: int, ny: int, nz: int, h: float):
    """Smallest and largest eigenvalue of the 7-point Dirichlet -Delta_h.

    Along one axis with n interior points the eigenvalues are (4/h^2) sin^2(k pi / (2(n+1))),
    k = 1..n (§7.1 gives the same modes as 2(1 - cos(.)) in its own scaling); the 3D
    operator is the Kronecker sum, so its extremes are the sums of the axis extremes.
    """
    lo = hi = 0.0
    for n in (nx, ny, nz):
        lo += 4.0 / (h * h) * math.sin(math.pi / (2.0 * (n + 1))) ** 2
        hi += 4.0 / (h * h) * math.sin(n * math.pi / (2.0 * (n + 1))) ** 2
    return lo, hi


def spectrum_box(op: Operator):
    """B = [b1, b2] x [-rho2, 0] containing every eigenvalue of A (Lemma 3.1 with Weyl).

    A = A1 - i A2 with A1 = s L_h - diag(m) and A2 = diag(a) >= 0.  By Weyl's inequality
    the Rayleigh quotient of A1 lies in [s*lmin - max m, s*lmax - min m] and that of A2 in
    [0, max a]; the Lemma's argument (lambda = v^H A v) then bounds every eigenvalue.
    """
    if op.kind == "spectral":
        lam = spectral_eigenvalues(op.nx, op.ny, op.nz, op.h)
        lo, hi = float(lam.min()), float(lam.max())
    else:
        lo, hi = laplacian_extremes(op.nx, op.ny, op.nz, op.h)
    b1 = op.s * lo - float(op.m.max())
    b2 = op.s * hi - float(op.m.min())
    rho2 = float(op.a.max())
    return b1, b2, rho2


def ellipse_quadrature(centre: complex, r: float, t: float, J: int, theta0: float):
    """Trapezoid rule on the ellipse centre + t r cos(theta) + i r sin(theta) (§6.1).

    (1/2 pi i) dz = (r cos theta + i t r sin theta) d theta / (2 pi), so J equispaced angles
    theta_j = theta0 + 2 pi (j-1)/J give weights sigma_j = (r cos theta_j + i t r sin theta_j)/J.
    """
    th = theta0 + 2.0 * math.pi * np.arange(J) / J
    z = centre + t * r * np.cos(th) + 1j * r * np.sin(th)
    sigma = (r * np.cos(th) + 1j * t * r * np.sin(th)) / J
    return z, sigma


def contour_nodes(J: int, t: float, eps: float, rho2: float):
    """Quadrature nodes z_j and weights sigma_j on the shifted ellipse (§6.2).

    phi = pi/J, r = (rho2/2 + eps)/sin(phi) (eq:quad-radius), centre -t r cos(phi) - i rho2/2,
    angles theta_j = (2j-1) phi, so that
    z_j = t r (cos theta_j - cos phi) + i (r sin theta_j - rho2/2)   (eq:quad-points).
    """
    phi = math.pi / J
    r = (rho2 / 2.0 + eps) / math.sin(phi)
    centre = complex(-t * r * math.cos(phi), -rho2 / 2.0)
    return ellipse_quadrature(centre, r, t, J, phi)


def quadrature_resolvent_sum(A: np.ndarray, z: np.ndarray, sigma: np.ndarray):
    """sum_j sigma_j/z_j (A - z_j I)^{-1} for a dense A: the quadrature of eq:rational."""
    n = A.shape[0]
    out = np.zeros((n, n), dtype=np.complex128)
    eye = np.eye(n)
    for zj, sj in zip(z, sigma):
        out += (sj / zj) * np.linalg.inv(A - zj * eye)
    return out


# ---------------------------------------------------------------------------------------
# Polynomial parameters (§4.2: eq:exp-taylor, eq:fix-pt-conv)
# ---------------------------------------------------------------------------------------

def ptilde(lam, q: int, delta: float, z0: complex):
    """Taylor polynomial of exp(-i delta (lam - z0)) of degree q (eq:exp-taylor)."""
    u = -1j * delta * (np.asarray(lam, dtype=np.complex128) - z0)
    term = np.ones_like(u)
    total = np.ones_like(u)
    for j in range(1, q + 1):
        term = term * u / j
        total = total + term
    return total


def box_boundary(b1: float, b2: float, rho2: float, per_side: int = 256) -> np.ndarray:
    """Points on the boundary of B: each of the 4 sides split into per_side equal pieces."""
    t = np.arange(per_side) / per_side
    v = [complex(b1, 0.0), complex(b2, 0.0), complex(b2, -rho2), complex(b1, -rho2)]
    pts = [v[k] + (v[(k + 1) % 4] - v[k]) * t for k in range(4)]
    return np.concatenate(pts)


def nu_of(q: int, delta: float, z: complex, z0: complex, boundary: np.ndarray) -> float:
    """max over the sampled boundary of |ptilde(lam)| / |ptilde(z)| (the rate in eq:fix-pt-conv)."""
    return float(np.max(np.abs(ptilde(boundary, q, delta, z0)))
                 / abs(complex(ptilde(z, q, delta, z0))))


def optimize_delta(q: int, z: complex, z0: complex, boundary: np.ndarray,
                   ngrid: int = 512, tol: float = 1e-10):
    """delta minimising nu for fixed q (eq:fix-pt-conv).  The paper only calls this an
    easy low-dimensional optimisation.  Reading: sign(delta) = sign(Im z) (so that
    delta*Im(lam - z0) < 0 on B, §4.2); |delta| on a uniform grid of ngrid points over
    (0, 4(q+1)/W], W = max |lam - z0| on the boundary, then golden-section search on the
    bracket around the best grid point.
    """
    sgn = 1.0 if z.imag > 0 else -1.0
    W = float(np.max(np.abs(boundary - z0)))
    dmax = 4.0 * (q + 1) / W
    grid = dmax * np.arange(1, ngrid + 1) / ngrid
    vals = np.array([nu_of(q, sgn * d, z, z0, boundary) for d in grid])
    k = int(np.argmin(vals))
    lo = grid[k - 1] if k > 0 else 0.0
    hi = grid[k + 1] if k + 1 < ngrid else dmax
    invphi = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c = b - invphi * (b - a)
    d = a + invphi * (b - a)
    fc = nu_of(q, sgn * c, z, z0, boundary)
    fd = nu_of(q, sgn * d, z, z0, boundary)
    while b - a > tol * dmax:
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - invphi * (b - a)
            fc = nu_of(q, sgn * c, z, z0, boundary)
        else:
            a, c, fc = c, d, fd
            d = a + invphi * (b - a)
            fd = nu_of(q, sgn * d, z, z0, boundary)
    best = 0.5 * (a + b)
    nbest = nu_of(q, sgn * best, z, z0, boundary)
    if vals[k] < nbest:
        best, nbest = grid[k], float(vals[k])
    return sgn * best, nbest


@dataclass
class NodeParams:
    z: complex
    sigma: complex
    z0: complex
    delta: float
    q: int
    nu: float
    sweeps: int


def node_parameters(z: complex, sigma: complex, b1: float, b2: float, rho2: float,
                    qmax: int = 5, reduction: float = 5.0, per_side: int = 256) -> NodeParams:
    """Per-node scheme parameters (§4.2 heuristic; §7.3 Table tab:param).

    z0 = (b1+b2)/2 + i Im z.  For each q <= qmax the best delta and its rate nu; the sweep
    count is the smallest s with nu^s <= 1/reduction (the paper stops each shifted solve
    once the residual drops by 5).  Reading of "prefer the minimum nu^(1/q)": take the q
    with the fewest matrix-vector products q*s; ties go to the smaller q.
    """
    z0 = complex(0.5 * (b1 + b2), z.imag)
    bd = box_boundary(b1, b2, rho2, per_side)
    best = None
    for q in range(1, qmax + 1):
        delta, nu = optimize_delta(q, z, z0, bd)
        if not nu < 1.0:
            continue
        sweeps = max(1, int(math.ceil(math.log(reduction) / -math.log(nu))))
        cand = (q * sweeps, q, NodeParams(complex(z), complex(sigma), z0, delta, q, nu, sweeps))
        if best is None or cand[:2] < best[:2]:
            best = cand
    if best is None:
        raise ValueError(f"no polynomial order q <= {qmax} converges at node {z}")
    return best[2]


def setup_nodes(op: Operator, J: int, t: float, eps: float, qmax: int = 5,
                reduction: float = 5.0):
    """Bounds, contour and per-node parameters for an operator (the whole host set-up)."""
    b1, b2, rho2 = spectrum_box(op)
    z, sigma = contour_nodes(J, t, eps, rho2)
    nodes = [node_parameters(zj, sj, b1, b2, rho2, qmax, reduction) for zj, sj in zip(z, sigma)]
    return (b1, b2, rho2), nodes


# ---------------------------------------------------------------------------------------
# Polynomial fixed-point solve of (A - zI) y = f  (§4.2, eq:fix-pt-exp)
# ---------------------------------------------------------------------------------------

def poly_coefficients(z: complex, z0: complex, delta: float, q: int):
    """c_j = (-i delta (z - z0))^j / j!, j = 0..q, and ptilde(z) = sum_j c_j."""
    u = -1j * delta * (z - z0)
    c = [complex(u ** j / math.factorial(j)) for j in range(q + 1)]
    return c, sum(c)


def poly_solve(op: Operator, f: np.ndarray, node: NodeParams, sweeps: int | None = None,
               y0: np.ndarray | None = None) -> np.ndarray:
    """sweeps steps of eq:fix-pt-exp from y0 (default 0):

        k_1 = -i delta ((A - z0) y - f)
        k_j = (-i delta / j) ((A - z0) k_{j-1} - c_{j-1} f),  j = 2..q
        y  <- (y + k_1 + ... + k_q) / ptilde(z)
    """
    q, delta, z0 = node.q, node.delta, node.z0
    nsw = node.sweeps if sweeps is None else sweeps
    c, pz = poly_coefficients(node.z, z0, delta, q)
    f = np.asarray(f, dtype=np.complex128).reshape(op.shape)
    y = np.zeros(op.shape, dtype=np.complex128) if y0 is None else np.array(y0, dtype=np.complex128).reshape(op.shape)
    for _ in range(nsw):
        k = -1j * delta * (op.apply(y, z0) - f)
        acc = y + k
        for j in range(2, q + 1):
            k = (-1j * delta / j) * (op.apply(k, z0) - c[j - 1] * f)
            acc = acc + k
        y = acc / pz
    return y


# ---------------------------------------------------------------------------------------
# GMRES pieces: CGS2 Arnoldi, complex Givens least squares
# ---------------------------------------------------------------------------------------

def cgs2(V: list, w: np.ndarray):
    """Classical Gram-Schmidt twice: h = V^H w, w -= V h, repeated; returns (w, h1 + h2)."""
    h1 = np.array([np.vdot(v, w) for v in V])
    for hi, v in zip(h1, V):
        w = w - hi * v
    h2 = np.array([np.vdot(v, w) for v in V])
    for hi, v in zip(h2, V):
        w = w - hi * v
    return w, h1 + h2


def givens(a: complex, b: float):
    """Rotation (c real, s complex) with [c, s; -conj(s), c] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0 + 0.0j
    if a == 0.0:
        return 0.0, 1.0 + 0.0j
    r = math.hypot(abs(a), b)
    return abs(a) / r, (a / abs(a)) * b / r


class _LeastSquares:
    """Incremental QR of the (k+1) x k Hessenberg matrix by Givens rotations."""

    def __init__(self, beta: float, m: int):
        self.R = np.zeros((m + 1, m), dtype=np.complex128)
        self.g = np.zeros(m + 1, dtype=np.complex128)
        self.g[0] = beta
        self.cs = []
        self.k = 0

    def add_column(self, h: np.ndarray, hnext: float) -> float:
        """Append column (h, hnext) of H; return |g_{k+1}|, the residual estimate."""
        k = self.k
        col = np.zeros(k + 2, dtype=np.complex128)
        col[:k + 1] = h
        col[k + 1] = hnext
        for i, (c, s) in enumerate(self.cs):
            a, b = col[i], col[i + 1]
            col[i] = c * a + s * b
            col[i + 1] = -np.conj(s) * a + c * b
        c, s = givens(complex(col[k]), float(col[k + 1].real))
        col[k] = c * col[k] + s * col[k + 1]
        col[k + 1] = 0.0
        self.cs.append((c, s))
        self.R[:k + 2, k] = col
        gk = self.g[k]
        self.g[k] = c * gk
        self.g[k + 1] = -np.conj(s) * gk
        self.k = k + 1
        return float(abs(self.g[k + 1]))

    def solve(self) -> np.ndarray:
        """Back substitution R y = g for the k columns added so far."""
        k = self.k
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (self.g[i] - np.dot(self.R[i, i + 1:k], y[i + 1:k])) / self.R[i, i]
        return y


def gmres_cycle(apply, b: np.ndarray, k: int, breakdown: float = 1e-14):
    """One GMRES(k) cycle from x0 = 0: CGS2 Arnoldi, Givens; returns (x, residual estimate).

    Stops early only on a happy breakdown h_{j+1,j} <= breakdown * ||A v_j||.
    """
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return np.zeros_like(b), 0.0
    V = [b / beta]
    ls = _LeastSquares(beta, k)
    est = beta
    for j in range(k):
        w = apply(V[j])
        wn = float(np.linalg.norm(w))
        w, h = cgs2(V, w)
        hn = float(np.linalg.norm(w))
        est = ls.add_column(h, hn)
        if hn <= breakdown * wn:
            break
        V.append(w / hn)
    y = ls.solve()
    x = np.zeros_like(b)
    for yi, v in zip(y, V):
        x = x + yi * v
    return x, est


# ---------------------------------------------------------------------------------------
# ILU(0) of the 7-point Laplacian: the inner preconditioner of §6.3 (used for the finite-
# difference runs of §7.3)
# ---------------------------------------------------------------------------------------

def ilu0_pivots(nx: int, ny: int, nz: int, cs: float) -> np.ndarray:
    """Pivots d of the incomplete LU factorisation without fill of K = cs * (7-point stencil:
    6 on the diagonal, -1 for each neighbour inside the grid), natural order (x fastest).

    For the 7-point pattern the product of the factors only adds entries outside the pattern
    besides the diagonal, so ILU(0) is M = (D + L) D^{-1} (D + U) with L, U the strict lower
    and upper parts of K and d_p = K_pp - sum over the lower neighbours q of K_pq K_qp / d_q.
    The recursion runs point by point in natural order (plain loops)."""
    d = np.zeros((nz, ny, nx))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                v = 6.0 * cs
                if i > 0:
                    v -= cs * cs / d[k, j, i - 1]
                if j > 0:
                    v -= cs * cs / d[k, j - 1, i]
                if k > 0:
                    v -= cs * cs / d[k - 1, j, i]
                d[k, j, i] = v
    return d


def ilu0_apply(d: np.ndarray, cs: float, t: np.ndarray) -> np.ndarray:
    """z = M^{-1} t for M = (D + L) D^{-1} (D + U) of ilu0_pivots: (D + L) u = t forward, then
    (D + U) z = D u backward, i.e. u_p = (t_p + cs * sum of u over the lower neighbours) / d_p
    and z_p = u_p + (cs / d_p) * sum of z over the upper neighbours.  Each value depends only
    on earlier (later) points, so the sweeps take the hyperplanes i + j + k = const in turn,
    vectorised over each plane, which gives the same values as the point-by-point order."""
    nz, ny, nx = d.shape
    t = np.asarray(t, dtype=np.complex128).reshape(nz, ny, nx)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    S = I + J + K
    planes = [np.nonzero(S.ravel() == w)[0] for w in range(nx + ny + nz - 2)]
    u = np.zeros(nz * ny * nx, dtype=np.complex128)
    z = np.zeros_like(u)
    tf, df = t.ravel(), d.ravel()
    Ii, Jj, Kk = I.ravel(), J.ravel(), K.ravel()
    sy, sz = nx, nx * ny
    for pts in planes:
        acc = tf[pts].copy()
        for off, ok in ((1, Ii[pts] > 0), (sy, Jj[pts] > 0), (sz, Kk[pts] > 0)):
            q = pts[ok]
            acc[ok] += cs * u[q - off]
        u[pts] = acc / df[pts]
    for pts in reversed(planes):
        acc = np.zeros(len(pts), dtype=np.complex128)
        for off, ok in ((1, Ii[pts] < nx - 1), (sy, Jj[pts] < ny - 1), (sz, Kk[pts] < nz - 1)):
            q = pts[ok]
            acc[ok] += z[q + off]
        z[pts] = u[pts] + (cs / df[pts]) * acc
    return z.reshape(nz, ny, nx)


def ilu0_preconditioner(op: Operator):
    """M^{-1} for the normalised operator's Laplacian part s L_h (weight cs = s / h^2)."""
    cs = op.s / (op.h * op.h)
    d = ilu0_pivots(op.nx, op.ny, op.nz, cs)
    return lambda t: ilu0_apply(d, cs, t)


# ---------------------------------------------------------------------------------------
# Regularised inverse Laplacian: the inner preconditioner of the spectral runs (§7.3)
# ---------------------------------------------------------------------------------------

def invlap_preconditioner(op: Operator):
    """M^{-1} = F^H diag(1 / max(lambda_i, 1)) F with lambda_i the normalised eigenvalues of
    the spectral Laplacian, s times spectral_eigenvalues (eq:eig-Laplacian-spectral): the
    inverse of the Laplacian on the modes above 1, the identity on the ones below."""
    lam = op.s * spectral_eigenvalues(op.nx, op.ny, op.nz, op.h)
    mult = 1.0 / np.maximum(lam, 1.0)

    def apply(t):
        t = np.asarray(t, dtype=np.complex128).reshape(op.shape)
        return np.fft.ifftn(mult * np.fft.fftn(t))
    return apply


# ---------------------------------------------------------------------------------------
# FCI (§2, Algorithm 1) and flexible GMRES around it
# ---------------------------------------------------------------------------------------

def fci(op: Operator, r: np.ndarray, nodes: list, k_in: int, shifted_solve=None,
        inner_precond=None):
    """Algorithm 1 applied to r:

    1. y_j = (A - z_j I)^{-1} r, here by the polynomial scheme with the node's sweeps
       (``shifted_solve(node, r)`` may replace it, e.g. by an exact solve in tests);
    2. w = sum_j sigma_j / z_j y_j;
    3. d = argmin_d ||r - d A w|| = (Aw)^H r / ||Aw||^2;
    4. v from k_in GMRES steps on A v = r - d A w (x0 = 0); with ``inner_precond`` (a map t ->
       M^{-1} t, §6.3) the GMRES runs right-preconditioned on A M^{-1} and v = M^{-1} x;
    5. return v + d w.
    """
    r = np.asarray(r, dtype=np.complex128).reshape(op.shape)
    w = np.zeros(op.shape, dtype=np.complex128)
    for nd in nodes:
        y = poly_solve(op, r, nd) if shifted_solve is None else shifted_solve(nd, r)
        w = w + (nd.sigma / nd.z) * y
    Aw = op.apply(w)
    den = np.vdot(Aw, Aw)
    d = np.vdot(Aw, r) / den if den != 0 else 0.0
    g = r - d * Aw
    if inner_precond is None:
        v, _ = gmres_cycle(op.apply, g, k_in)
    else:
        x, _ = gmres_cycle(lambda q: op.apply(inner_precond(q)), g, k_in)
        v = inner_precond(x)
    return v + d * w


@dataclass
class SolveResult:
    u: np.ndarray
    cycles: int
    its: int
    rel_res_true: float
    converged: bool
    history: list


def fgmres(op: Operator, f: np.ndarray, precond, m: int, rtol: float, max_cycles: int,
           fixed_its: int = 0, breakdown: float = 1e-14) -> SolveResult:
    """Right-preconditioned flexible GMRES(m) (Saad's FGMRES), x0 = 0.

    Per step: z_k = precond(v_k); w = A z_k; CGS2; Givens.  A cycle ends after m steps,
    on a happy breakdown, or (unless fixed_its > 0) when the Givens estimate drops to
    rtol*||f||; then x += Z y and the true residual ||f - A x||/||f|| is recomputed.
    Convergence is declared on the true residual only.  With fixed_its > 0 exactly that
    many steps are taken (cycles of m), regardless of rtol: the deterministic mode used
    to compare iterates.
    """
    f = np.asarray(f, dtype=np.complex128).reshape(op.shape)
    fn = float(np.linalg.norm(f))
    x = np.zeros(op.shape, dtype=np.complex128)
    its = 0
    hist = []
    if fn == 0.0:
        return SolveResult(x, 0, 0, 0.0, True, hist)
    cycles = 0
    rel = 1.0
    while cycles < max_cycles:
        r = f - op.apply(x)
        beta = float(np.linalg.norm(r))
        rel = beta / fn
        hist.append(rel)
        if fixed_its > 0:
            if its >= fixed_its:
                break
        elif rel <= rtol:
            break
        cycles += 1
        V = [r / beta]
        Z = []
        ls = _LeastSquares(beta, m)
        for _ in range(m):
            zk = precond(V[-1])
            Z.append(zk)
            w = op.apply(zk)
            wn = float(np.linalg.norm(w))
            w, h = cgs2(V, w)
            hn = float(np.linalg.norm(w))
            est = ls.add_column(h, hn)
            its += 1
            if hn <= breakdown * wn:
                break
            V.append(w / hn)
            if fixed_its > 0:
                if its >= fixed_its:
                    break
            elif est <= rtol * fn:
                break
        y = ls.solve()
        for yi, zk in zip(y, Z):
            x = x + yi * zk
    r = f - op.apply(x)
    rel = float(np.linalg.norm(r)) / fn
    if not hist or hist[-1] != rel:
        hist.append(rel)
    return SolveResult(x, cycles, its, rel, rel <= rtol, hist)


def solve(op: Operator, f: np.ndarray, nodes: list, m: int, k_in: int, rtol: float,
          max_cycles: int, fixed_its: int = 0, inner_precond=None) -> SolveResult:
    """A u = f by FGMRES(m) preconditioned with FCI (Algorithm 1)."""
    return fgmres(op, f, lambda v: fci(op, v, nodes, k_in, inner_precond=inner_precond), m,
                  rtol, max_cycles, fixed_its)


# ---------------------------------------------------------------------------------------
# Case Two (§3, eq:mat-2x2, Theorem thm:spectrum-2x2): the double-size system
# ---------------------------------------------------------------------------------------

@dataclass
class Operator2x2:
    """Case Two's coefficient matrix iC - I on stacked fields x = (x1; x2) of shape
    (2, nz, ny, nx), with C = [[0, I], [-(A1 + I), -A2]] (eq:mat-2x2) and A = A1 - i A2 the
    Case One operator split as in spectrum_box: A1 = s L_h - diag(m) Hermitian, A2 =
    diag(a) positive semi-definite.  (iC - I)(iu; u) = (0; f) holds exactly when A u = f.
    It exposes the ``apply`` / ``shape`` interface the polynomial scheme, Algorithm 1 and
    FGMRES use, so those run on it unchanged.
    """
    base: Operator

    @property
    def shape(self):
        return (2,) + self.base.shape

    @property
    def n(self):
        return 2 * self.base.n

    def apply_c(self, x: np.ndarray):
        """C x = (x2; -(A1 + I) x1 - A2 x2)."""
        x = np.asarray(x, dtype=np.complex128).reshape(self.shape)
        x1, x2 = x[0], x[1]
        a1x1 = self.base.apply(x1) + 1j * self.base.a * x1  # A1 x1 = A x1 + i A2 x1
        return np.stack([x2, -(a1x1 + x1) - self.base.a * x2])

    def apply(self, x: np.ndarray, z: complex = 0.0) -> np.ndarray:
        """((iC - I) - z I) x."""
        x = np.asarray(x, dtype=np.complex128).reshape(self.shape)
        return 1j * self.apply_c(x) - x - z * x


def spectrum_box_2x2(op: Operator):
    """A rectangle [b1, b2] x [-rho2, 0] containing the spectrum of iC - I.

    The Remark after Theorem thm:spectrum-2x2 puts it in |mu + 1| <= R, -rho2 <= Im mu <= 0,
    R = rho2/2 + sqrt(rho2^2/4 + rho1), with rho1 = rho(A1 + I) and rho2 = rho(A2) as in
    Lemma lem:spectrum-1x1.  Reading: rho1 from Weyl's inequality as in spectrum_box,
    rho(A1 + I) <= s*lmax - min m + 1 (A1 + I is positive semi-definite since m <= 1), and
    [b1, b2] = [-1 - R, -1 + R].  Returns (b1, b2, rho2, rho1, R).
    """
    _, hi = laplacian_extremes(op.nx, op.ny, op.nz, op.h)
    rho1 = op.s * hi - float(op.m.min()) + 1.0
    rho2 = float(op.a.max())
    R = rho2 / 2.0 + math.sqrt(rho2 * rho2 / 4.0 + rho1)
    return -1.0 - R, -1.0 + R, rho2, rho1, R


def setup_nodes_2x2(op: Operator, J: int, t: float, eps: float, qmax: int = 5,
                    reduction: float = 5.0):
    """Contour and per-node parameters of Algorithm 1 for iC - I: the nodes of eq:quad-points
    depend on rho2 and eps only, the polynomial scheme's rate on the rectangle above."""
    b1, b2, rho2, _, _ = spectrum_box_2x2(op)
    z, sigma = contour_nodes(J, t, eps, rho2)
    nodes = [node_parameters(zj, sj, b1, b2, rho2, qmax, reduction) for zj, sj in zip(z, sigma)]
    return (b1, b2, rho2), nodes


def solve_2x2(op: Operator, f: np.ndarray, nodes: list, m: int, k_in: int, rtol: float,
              max_cycles: int, fixed_its: int = 0) -> SolveResult:
    """Case Two: (iC - I) Y = (0; f) by FGMRES(m) with FCI on iC - I; the solution of
    A u = f is u = Y[1] (eq:mat-2x2).  rel_res_true is the 2x2 system's residual."""
    op2 = Operator2x2(op)
    F = np.stack([np.zeros(op.shape, dtype=np.complex128),
                  np.asarray(f, dtype=np.complex128).reshape(op.shape)])
    return fgmres(op2, F, lambda v: fci(op2, v, nodes, k_in), m, rtol, max_cycles, fixed_its)
