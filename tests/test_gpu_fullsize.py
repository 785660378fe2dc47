"""Parity at the benchmark's full sizes, in the configuration bench.py times, checked with
properties the oracle computes cheaply at any size: the float64 true residual of every GPU
solution (one oracle matvec each), the stencil itself on 256^3 fields, and the 256^3
sixteen-source configuration solved to 1e-8.

Tolerances: the solver's own 1e-8 relative residual (plus 1e-12 for the difference between the
library's and numpy's float64 residual sums); stencil float64 1e-14, complex64 2e-6 relative L2.
"""
import numpy as np
import pytest

import workloads as W
from oracle import hz_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1811_12378_gb300 as hzpkg  # noqa: E402

DEV = "cuda:0"


def _residual(op, f, u):
    sf = op.s * f
    return float(np.linalg.norm(sf - op.apply(u)) / np.linalg.norm(sf))


@pytest.mark.parametrize("prec", [hzpkg.HZ_MIXED_C64, hzpkg.HZ_MIXED_C64_FF,
                                  hzpkg.HZ_MIXED_C64_FCI32, hzpkg.HZ_C128])
def test_gaussian_bumps_64_solution_residual(prec):
    """The benchmark solve (64^3, J = 8, FGMRES(30), 1e-8) in every precision form."""
    wl = W.gaussian_bumps_64()
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    with hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                       nrhs_max=1, restart_max=wl.restart, inner_k_max=wl.k_in) as P:
        f = torch.from_numpy(wl.f.reshape(1, -1).copy()).to(DEV)
        u, st = P.solve(f, restart=wl.restart, inner_k=wl.k_in, rtol=wl.rtol, max_cycles=20,
                        precision=prec)
    assert st[0].converged
    res = _residual(op, wl.f[0], u.cpu().numpy().reshape(op.shape))
    assert res <= wl.rtol + 1e-12
    assert abs(res - st[0].rel_res_true) <= 1e-10


def test_uneven_batch_solution_residuals():
    """All 48 right-hand sides of the 12-instance uneven batch (48^3, 64^3, 96^3)."""
    wls = W.layered_batch()
    probs = [hzpkg.Problem(w.c, w.h, w.omega, w.layer_cells, w.sigma_max, w.J, w.t, w.eps,
                           nrhs_max=w.nrhs, restart_max=w.restart, inner_k_max=w.k_in)
             for w in wls]
    try:
        fs = [torch.from_numpy(w.f.reshape(w.nrhs, -1).copy()).to(DEV) for w in wls]
        us, sts = hzpkg.solve_batched(probs, fs, restart=30, inner_k=4, rtol=1e-8,
                                      max_cycles=30, precision=hzpkg.HZ_MIXED_C64_FCI32)
        for w, u, st in zip(wls, us, sts):
            op = O.make_operator(w.c, w.h, w.omega, w.layer_cells, w.sigma_max)
            un = u.cpu().numpy().reshape((w.nrhs,) + op.shape)
            for v in range(w.nrhs):
                assert st[v].converged
                assert _residual(op, w.f[v], un[v]) <= 1e-8 + 1e-12
    finally:
        for P in probs:
            P.close()


def test_stencil_256():
    """(A - zI)x on 256^3 fields (the large-grid configuration), both precisions."""
    N = 256
    h = 1.0 / (N + 1)
    c = W.medium_gaussian_bumps(1, N, N, N, h)
    om = W.omega_for_ppw(c, h, 8.0)
    op = O.make_operator(c, h, om, 12, 1.0)
    x = W.random_field(8, 1, N, N, N)[0]
    z = 0.3 - 1.0j
    ref = op.apply(x, z)
    with hzpkg.Problem(c, h, om, 12, 1.0, 1, 1.0, 0.25, nrhs_max=1, restart_max=1,
                       inner_k_max=0) as P:
        xd = torch.from_numpy(x.reshape(1, -1)).to(DEV)
        y = P.apply_shifted(xd, z).cpu().numpy().reshape(op.shape)
        assert np.linalg.norm(y - ref) <= 1e-14 * np.linalg.norm(ref)
        y32 = P.apply_shifted(xd.to(torch.complex64), z).cpu().numpy().reshape(op.shape)
        assert np.linalg.norm(y32 - ref) <= 2e-6 * np.linalg.norm(ref)


def test_large_256_sixteen_sources_to_1e8():
    """The large configuration at full size (256^3, c in [1, 3], 12-cell sponge, 8 ppw, J = 8,
    FGMRES(40), 16 point sources) solved to a float64 true residual of 1e-8 in the float64-outer
    mixed form, as two calls of 8 right-hand sides with complex64 sweep workspace and
    complex64-stored directions (16 at once would not fit in the device memory).  Every
    reported true residual must be at most 1e-8 and equal the oracle's own matvec residual of
    the returned solution."""
    wl, idx = W.large_bumps_256()
    N = wl.nx
    n = N ** 3
    amp = 1.0 / wl.h ** 3
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    with hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                       nrhs_max=8, restart_max=wl.restart, inner_k_max=wl.k_in,
                       flags=hzpkg.HZ_LIMIT_SWEEPS_C64 | hzpkg.HZ_LIMIT_Z_C64) as P:
        for half in range(2):
            srcs = idx[8 * half: 8 * half + 8]
            f = torch.zeros((8, n), dtype=torch.complex128, device=DEV)
            for r, (i, j, k) in enumerate(srcs):
                f[r, i + N * (j + N * k)] = amp
            u, st = P.solve(f, restart=wl.restart, inner_k=wl.k_in, rtol=wl.rtol, max_cycles=12,
                            precision=hzpkg.HZ_MIXED_C64)
            del f
            for r, (i, j, k) in enumerate(srcs):
                assert st[r].converged and st[r].rel_res_true <= wl.rtol, (r, st[r])
                fr = np.zeros(op.shape, dtype=np.complex128)
                fr[k, j, i] = amp
                ur = u[r].cpu().numpy().reshape(op.shape)
                res = _residual(op, fr, ur)
                assert res <= wl.rtol + 1e-12
                assert abs(res - st[r].rel_res_true) <= 1e-12 + 1e-9 * res
            del u
