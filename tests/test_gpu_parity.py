"""GPU parity: every call of the C ABI against the CPU oracle on the same seeded inputs.

Sizes span several 32x4 stencil tiles with ragged tails in x and y, 1x1x1 and degenerate
grids, several right-hand sides per launch, and the full 64^3 Gaussian-bump workload.
Tolerances (relative L2): float64 stencil 1e-14, float64 polynomial solve 1e-12, float64
FCI 1e-11, float64 FGMRES iterates at a fixed step count 1e-9; complex64 stencil 2e-6,
complex64 polynomial solve / mixed FCI 1e-5 (float32 rounding, about 1e-7 a step, through
contracting iterations).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import hz_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1811_12378_gb300 as hzpkg  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV).to(dtype).contiguous()


def to_np(t):
    return t.detach().cpu().numpy()


def oracle_of(wl):
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    (b1, b2, rho2), nodes = O.setup_nodes(op, wl.J, wl.t, wl.eps)
    return op, nodes


def problem_of(wl, nodes=None, nrhs_max=4, restart_max=30, inner_k_max=8):
    P = hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                      nrhs_max=nrhs_max, restart_max=restart_max, inner_k_max=inner_k_max)
    if nodes is not None:
        P.set_nodes([nd.z for nd in nodes], [nd.sigma for nd in nodes], [nd.z0 for nd in nodes],
                    [nd.delta for nd in nodes], [nd.q for nd in nodes],
                    [nd.sweeps for nd in nodes])
    return P


RAGGED = [((37, 19, 11), 3), ((33, 5, 2), 1), ((64, 64, 64), 8), ((1, 1, 1), 0), ((2, 7, 1), 1)]


@pytest.mark.parametrize("shape,layer", RAGGED, ids=lambda v: str(v))
def test_stencil_parity(shape, layer):
    """(A - zI)x for 3 fields per launch, float64 and float32 paths (§7.1)."""
    nx, ny, nz = shape
    wl = W.small_case(11, nx, ny, nz, layer=layer, medium="bumps" if nx > 1 else "const")
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    x = W.random_field(5, 3, nx, ny, nz)
    with hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, 4, 1.0, 1.0) as P:
        for z in (0.0, 0.3 - 1.7j, -2.0 + 0.5j):
            ref = np.stack([op.apply(x[v], z) for v in range(3)])
            y = to_np(P.apply_shifted(to_dev(x), z))
            assert rel(y, ref) <= 1e-14
            y32 = to_np(P.apply_shifted(to_dev(x, torch.complex64), z))
            assert rel(y32, ref) <= 2e-6


@pytest.mark.parametrize("shape,layer", [((37, 19, 11), 3), ((2, 7, 1), 1), ((1, 1, 1), 0)],
                         ids=lambda v: str(v))
def test_case_two_operator_parity(shape, layer):
    """Case Two (§3 eq:mat-2x2): ((iC - I) - zI) x on 2 vectors of two stacked fields each,
    against the oracle's Operator2x2 (pinned on CPU by the dense block matrix and Theorem
    thm:spectrum-2x2), float64 and float32 paths, the unshifted and two shifted forms."""
    nx, ny, nz = shape
    wl = W.small_case(12, nx, ny, nz, layer=layer, medium="bumps" if nx > 1 else "const")
    op2 = O.Operator2x2(O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max))
    x = W.random_field(13, 4, nx, ny, nz).reshape(2, 2, nz, ny, nx)
    with hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, 4, 1.0, 1.0) as P:
        for z in (0.0, 0.3 - 0.7j, -1.5 + 0.2j):
            ref = np.stack([op2.apply(x[v], z) for v in range(2)])
            y = to_np(P.apply_2x2(to_dev(x.reshape(2, -1)), z))
            assert rel(y, ref) <= 1e-14
            y32 = to_np(P.apply_2x2(to_dev(x.reshape(2, -1), torch.complex64), z))
            assert rel(y32, ref) <= 2e-6


def test_stencil_sine_modes_gpu():
    """P1 on the GPU: sine modes are eigenvectors of the stencil with c = 1, no sponge."""
    nx, ny, nz = 40, 21, 9
    h = 1.0 / 41
    c = np.ones((nz, ny, nx))
    omega = 2 * math.pi / (8 * h)
    s = 1.0 / omega ** 2
    with hzpkg.Problem(c, h, omega, 0, 0.0, 4, 1.0, 1.0) as P:
        for kx, ky, kz in [(1, 1, 1), (7, 20, 3), (40, 2, 9)]:
            i = np.arange(1, nx + 1)
            j = np.arange(1, ny + 1)
            k = np.arange(1, nz + 1)
            v = (np.sin(kz * np.pi * k / (nz + 1))[:, None, None]
                 * np.sin(ky * np.pi * j / (ny + 1))[None, :, None]
                 * np.sin(kx * np.pi * i / (nx + 1))[None, None, :]).astype(np.complex128)
            lam = sum(4 / h ** 2 * math.sin(kk * math.pi / (2 * (nn + 1))) ** 2
                      for kk, nn in ((kx, nx), (ky, ny), (kz, nz)))
            mu = s * lam - 1.0
            y = to_np(P.apply_shifted(to_dev(v[None])))[0]
            scale = 12 / h ** 2 * s + 1.0   # bound of |A| on the grid
            assert np.linalg.norm(y - mu * v) <= 1e-14 * scale * np.linalg.norm(v)


@pytest.mark.parametrize("prec", [hzpkg.HZ_C128, hzpkg.HZ_MIXED_C64])
def test_shifted_solve_parity(prec):
    """Each node's polynomial solve (eq:fix-pt-exp) on 2 right-hand sides at once."""
    wl = W.small_case(3, 13, 9, 7, layer=2, J=4)
    op, nodes = oracle_of(wl)
    f = W.random_field(17, 2, wl.nx, wl.ny, wl.nz)
    dt = torch.complex128 if prec == hzpkg.HZ_C128 else torch.complex64
    tol = 1e-12 if prec == hzpkg.HZ_C128 else 1e-5
    with problem_of(wl, nodes) as P:
        for j, nd in enumerate(nodes):
            y = to_np(P.shifted_solve(j, to_dev(f, dt), precision=prec))
            ref = np.stack([O.poly_solve(op, f[v], nd) for v in range(2)])
            assert rel(y, ref) <= tol, (j, nd.q, nd.sweeps)


def test_shifted_solve_q1_and_high_order():
    """Orders 1 (ping-pong of y) and 5 through hz_problem_set_nodes."""
    wl = W.small_case(8, 10, 6, 5, layer=1, J=3)
    op, nodes = oracle_of(wl)
    b1, b2, rho2 = O.spectrum_box(op)
    custom = []
    for nd, q, sw in zip(nodes, (1, 5, 2), (7, 2, 3)):
        d, nu = O.optimize_delta(q, nd.z, nd.z0, O.box_boundary(b1, b2, rho2))
        custom.append(O.NodeParams(nd.z, nd.sigma, nd.z0, d, q, nu, sw))
    f = W.random_field(2, 1, wl.nx, wl.ny, wl.nz)
    with problem_of(wl, custom) as P:
        for j, nd in enumerate(custom):
            y = to_np(P.shifted_solve(j, to_dev(f)))
            assert rel(y[0], O.poly_solve(op, f[0], nd)) <= 1e-12


@pytest.mark.parametrize("prec,kin", [(hzpkg.HZ_C128, 3), (hzpkg.HZ_C128, 0),
                                      (hzpkg.HZ_MIXED_C64, 4), (hzpkg.HZ_MIXED_C64_FCI32, 4),
                                      (hzpkg.HZ_MIXED_C64_FCI32, 0),
                                      (hzpkg.HZ_MIXED_C64_FCI32, 10)])
def test_fci_parity(prec, kin):
    """Algorithm 1 on 3 fields at once (k_in = 0 and 10 cover the edges of the inner solve)."""
    wl = W.small_case(6, 23, 10, 9, layer=2, J=5)
    op, nodes = oracle_of(wl)
    r = W.random_field(9, 3, wl.nx, wl.ny, wl.nz)
    with problem_of(wl, nodes, inner_k_max=10) as P:
        out = to_np(P.fci(to_dev(r), inner_k=kin, precision=prec))
    ref = np.stack([O.fci(op, r[v], nodes, kin) for v in range(3)])
    tol = {hzpkg.HZ_C128: 1e-11, hzpkg.HZ_MIXED_C64: 1e-5, hzpkg.HZ_MIXED_C64_FCI32: 2e-5}[prec]
    assert rel(out, ref) <= tol


@pytest.mark.parametrize("kin", [0, 1, 4, 10])
def test_fci_fused_tail_one_rhs(kin):
    """Steps 3-5 of Algorithm 1 for one right-hand side as one cooperative kernel (k_in up to 4
    and up to 16 use different instances), with h_{j+1,j} from the Pythagorean difference (the
    default) or summed: against the oracle, and against the per-piece kernels, which differ
    from it only in float32 rounding; deterministic."""
    wl = W.small_case(16, 22, 13, 9, layer=2, J=5)
    op, nodes = oracle_of(wl)
    r = W.random_field(19, 1, wl.nx, wl.ny, wl.nz)
    with problem_of(wl, nodes, nrhs_max=1, inner_k_max=10) as P:
        fused = to_np(P.fci(to_dev(r), inner_k=kin, precision=hzpkg.HZ_MIXED_C64_FCI32))
        fused2 = to_np(P.fci(to_dev(r), inner_k=kin, precision=hzpkg.HZ_MIXED_C64_FCI32))
        P.fused_tail(2)  # the norm after the second Gram-Schmidt pass always summed
        summed = to_np(P.fci(to_dev(r), inner_k=kin, precision=hzpkg.HZ_MIXED_C64_FCI32))
        P.fused_tail(False)
        piece = to_np(P.fci(to_dev(r), inner_k=kin, precision=hzpkg.HZ_MIXED_C64_FCI32))
        with pytest.raises(hzpkg.HzError):
            P.fused_tail(-1)
    ref = O.fci(op, r[0], nodes, kin)
    assert np.array_equal(fused, fused2)
    for out in (fused, summed):
        assert rel(out[0], ref) <= 2e-5
        assert rel(out[0], piece[0]) <= 2e-5


def test_fci_eigenvector_exact_gpu():
    """P7 through the GPU: FCI of a sine mode returns v / mu."""
    nx, ny, nz = 6, 5, 7
    h = 1.0 / 8
    c = np.ones((nz, ny, nx))
    omega = 2 * math.pi / (6 * h)
    with hzpkg.Problem(c, h, omega, 0, 0.0, 4, 1.0, 0.5) as P:
        i, j, k = np.arange(1, nx + 1), np.arange(1, ny + 1), np.arange(1, nz + 1)
        v = (np.sin(2 * np.pi * k / (nz + 1))[:, None, None]
             * np.sin(1 * np.pi * j / (ny + 1))[None, :, None]
             * np.sin(3 * np.pi * i / (nx + 1))[None, None, :]).astype(np.complex128)
        lam = sum(4 / h ** 2 * math.sin(kk * math.pi / (2 * (nn + 1))) ** 2
                  for kk, nn in ((3, nx), (1, ny), (2, nz)))
        mu = lam / omega ** 2 - 1.0
        out = to_np(P.fci(to_dev(v[None]), inner_k=3))[0]
        assert rel(out, v / mu) <= 1e-12


def test_fci_full_size_gaussian_bumps_64():
    """FCI at the full 64^3, J = 8 Gaussian-bump workload: float64 and mixed forms."""
    wl = W.gaussian_bumps_64()
    op, nodes = oracle_of(wl)
    r = W.random_field(4, 1, wl.nx, wl.ny, wl.nz)
    ref = O.fci(op, r[0], nodes, wl.k_in)
    with problem_of(wl, nodes, nrhs_max=1, restart_max=30, inner_k_max=4) as P:
        out = to_np(P.fci(to_dev(r), inner_k=wl.k_in))
        assert rel(out[0], ref) <= 1e-11
        outm = to_np(P.fci(to_dev(r), inner_k=wl.k_in, precision=hzpkg.HZ_MIXED_C64))
        assert rel(outm[0], ref) <= 1e-5
        out32 = to_np(P.fci(to_dev(r), inner_k=wl.k_in, precision=hzpkg.HZ_MIXED_C64_FCI32))
        assert rel(out32[0], ref) <= 2e-5


def test_solve_fixed_iterations_parity():
    """FGMRES(5) iterates across two restarts equal the oracle's at a fixed step count."""
    wl = W.small_case(3, 13, 9, 7, layer=2, J=4)
    op, nodes = oracle_of(wl)
    f = wl.f[0]
    res = O.solve(op, op.s * f, nodes, m=5, k_in=3, rtol=1e-30, max_cycles=100, fixed_its=12)
    with problem_of(wl, nodes, nrhs_max=1, restart_max=5, inner_k_max=3) as P:
        u, st = P.solve(to_dev(f[None]), restart=5, inner_k=3, rtol=1e-30, max_cycles=100,
                        fixed_its=12)
    assert st[0].its == 12 and st[0].cycles == 3 == res.cycles
    assert rel(to_np(u)[0], res.u) <= 1e-9
    assert st[0].rel_res_true == pytest.approx(res.rel_res_true, rel=1e-6)


def test_solve_point_source_32_converges_like_oracle():
    """32^3 point source (c = 1, 10 ppw, J = 4): float64 FGMRES(30) reaches 1e-8 in the
    oracle's step count; at that fixed count the iterates agree; the true residual is checked
    with the oracle's operator."""
    wl = W.point_source_32()
    op, nodes = oracle_of(wl)
    f = wl.f[0]
    res = O.solve(op, op.s * f, nodes, m=30, k_in=4, rtol=1e-8, max_cycles=20)
    with problem_of(wl, nodes, nrhs_max=1, restart_max=30, inner_k_max=4) as P:
        u, st = P.solve(to_dev(f[None]), restart=30, inner_k=4, rtol=1e-8, max_cycles=20)
        uf, stf = P.solve(to_dev(f[None]), restart=30, inner_k=4, rtol=1e-30, max_cycles=20,
                          fixed_its=res.its)
    assert st[0].converged and res.converged
    assert abs(st[0].its - res.its) <= 1
    ug = to_np(u)[0]
    true = np.linalg.norm(op.s * f - op.apply(ug)) / np.linalg.norm(op.s * f)
    assert true <= 1e-8
    assert rel(to_np(uf)[0], res.u) <= 1e-9


@pytest.mark.parametrize("prec", [hzpkg.HZ_MIXED_C64, hzpkg.HZ_MIXED_C64_FCI32,
                                  hzpkg.HZ_MIXED_C64_FF])
def test_mixed_solve_point_source_32(prec):
    """Mixed forms (complex64 sweeps, or the whole FCI in complex64; float64 outer Krylov and
    residual) reach the same 1e-8 true residual in about the float64 step count."""
    wl = W.point_source_32()
    op, nodes = oracle_of(wl)
    f = wl.f[0]
    with problem_of(wl, nodes, nrhs_max=1, restart_max=30, inner_k_max=4) as P:
        u64, s64 = P.solve(to_dev(f[None]), restart=30, inner_k=4, rtol=1e-8, max_cycles=20)
        u32, s32 = P.solve(to_dev(f[None]), restart=30, inner_k=4, rtol=1e-8, max_cycles=20,
                           precision=prec)
    assert s32[0].converged
    ug = to_np(u32)[0]
    true = np.linalg.norm(op.s * f - op.apply(ug)) / np.linalg.norm(op.s * f)
    assert true <= 1e-8
    assert s32[0].its <= 1.25 * s64[0].its + 2


def test_float_pair_arnoldi_matches_float64_arnoldi():
    """HZ_MIXED_C64_FF differs from HZ_MIXED_C64_FCI32 only in the arithmetic of the outer
    Arnoldi (float pairs, about 48 bits, against float64) and shares its complex64 FCI, so at
    a fixed number of outer steps (two restart cycles) the iterates agree to near float64
    rounding; 2 right-hand sides, ragged grid."""
    wl = W.small_case(41, 13, 10, 9, nrhs=2, layer=2, J=4)
    op, nodes = oracle_of(wl)
    with problem_of(wl, nodes, nrhs_max=2, restart_max=6, inner_k_max=3) as P:
        kw = dict(restart=6, inner_k=3, rtol=1e-30, max_cycles=3, fixed_its=11)
        u64, s64 = P.solve(to_dev(wl.f), precision=hzpkg.HZ_MIXED_C64_FCI32, **kw)
        uff, sff = P.solve(to_dev(wl.f), precision=hzpkg.HZ_MIXED_C64_FF, **kw)
    assert [s.its for s in sff] == [s.its for s in s64] == [11, 11]
    for v in range(2):
        assert rel(to_np(uff)[v], to_np(u64)[v]) <= 1e-10
        assert abs(sff[v].rel_res_true - s64[v].rel_res_true) <= 1e-10 * max(
            s64[v].rel_res_true, 1e-300) + 1e-14


@pytest.mark.parametrize("restart", [5, 12])
def test_float_pair_arnoldi_fused_one_rhs(restart):
    """One right-hand side: the outer float-pair Arnoldi step as one cooperative kernel (the
    default, h_{k+1,k} from the Pythagorean difference) against the same kernel summing the
    last norm, against its five-kernel form, which has the same per-point arithmetic and groups
    the global float-pair sums differently, and against the float64 outer Arnoldi; a fixed
    number of outer steps over three cycles (restart 12: basis counts past one group of 8),
    ragged grid; the cooperative form is deterministic."""
    wl = W.small_case(43, 13, 10, 9, nrhs=1, layer=2, J=4)
    op, nodes = oracle_of(wl)
    its = 2 * restart + 1
    with problem_of(wl, nodes, nrhs_max=1, restart_max=restart, inner_k_max=3) as P:
        kw = dict(restart=restart, inner_k=3, rtol=1e-30, max_cycles=3, fixed_its=its)
        ua, sa = P.solve(to_dev(wl.f), precision=hzpkg.HZ_MIXED_C64_FF, **kw)
        ub, sb = P.solve(to_dev(wl.f), precision=hzpkg.HZ_MIXED_C64_FF, **kw)
        P.fused_arnoldi(2)  # the same kernel with the last norm always summed
        ue, se = P.solve(to_dev(wl.f), precision=hzpkg.HZ_MIXED_C64_FF, **kw)
        P.fused_arnoldi(False)
        uc, sc = P.solve(to_dev(wl.f), precision=hzpkg.HZ_MIXED_C64_FF, **kw)
        ud, sd = P.solve(to_dev(wl.f), precision=hzpkg.HZ_MIXED_C64_FCI32, **kw)
        with pytest.raises(hzpkg.HzError):
            P.fused_arnoldi(3)
    assert [s.its for s in (sa[0], sb[0], sc[0], sd[0], se[0])] == [its] * 5
    assert np.array_equal(to_np(ua), to_np(ub))
    for u, st in ((uc, sc), (ud, sd), (ue, se)):
        assert rel(to_np(ua)[0], to_np(u)[0]) <= 1e-10
        # a 1e-10 relative change of u moves r = s f - A u by up to ||A|| ||u|| 1e-10, about
        # the condition number (here ~1e3) times 1e-10 relative to ||s f||
        assert abs(sa[0].rel_res_true - st[0].rel_res_true) <= 1e-7 * st[0].rel_res_true + 1e-13


def test_batched_rhs_equal_single_solves():
    """Several right-hand sides in one call give the results of separate calls."""
    wl = W.small_case(12, 12, 11, 10, nrhs=3, layer=2, J=4)
    op, nodes = oracle_of(wl)
    with problem_of(wl, nodes, nrhs_max=3, restart_max=8, inner_k_max=3) as P:
        ub, sb = P.solve(to_dev(wl.f), restart=8, inner_k=3, rtol=1e-9, max_cycles=30)
        for v in range(3):
            u1, s1 = P.solve(to_dev(wl.f[v:v + 1]), restart=8, inner_k=3, rtol=1e-9,
                             max_cycles=30)
            assert s1[0].its == sb[v].its
            assert rel(to_np(ub)[v], to_np(u1)[0]) <= 1e-14
            true = np.linalg.norm(op.s * wl.f[v] - op.apply(to_np(ub)[v])) / np.linalg.norm(
                op.s * wl.f[v])
            assert true <= 1e-9


def test_solve_batched_equals_single_solves():
    """hz_solve_batched over problems of different shapes and media (2 right-hand sides each)
    reproduces separate hz_solve calls exactly; true residuals checked with the oracle."""
    wls = [W.small_case(21, 10, 9, 8, nrhs=2, layer=2, J=4),
           W.small_case(22, 12, 12, 12, nrhs=2, layer=2, J=5, medium="layered"),
           W.small_case(23, 7, 11, 9, nrhs=2, layer=1, J=3)]
    probs = [problem_of(w, None, nrhs_max=2, restart_max=8, inner_k_max=3) for w in wls]
    try:
        fs = [to_dev(w.f) for w in wls]
        for prec in (hzpkg.HZ_C128, hzpkg.HZ_MIXED_C64_FCI32, hzpkg.HZ_MIXED_C64_FF):
            us, sts = hzpkg.solve_batched(probs, fs, restart=8, inner_k=3, rtol=1e-9,
                                          max_cycles=40, precision=prec)
            for P, w, f, u, st in zip(probs, wls, fs, us, sts):
                u1, s1 = P.solve(f, restart=8, inner_k=3, rtol=1e-9, max_cycles=40,
                                 precision=prec)
                assert [x.its for x in st] == [x.its for x in s1]
                assert np.array_equal(to_np(u), to_np(u1))
                op = O.make_operator(w.c, w.h, w.omega, w.layer_cells, w.sigma_max)
                for v in range(2):
                    sf = op.s * w.f[v]
                    assert np.linalg.norm(sf - op.apply(to_np(u)[v])) <= 1e-9 * np.linalg.norm(sf)
    finally:
        for P in probs:
            P.close()


def test_edge_cases():
    wl = W.small_case(1, 4, 3, 2, layer=1, J=2)
    with problem_of(wl, None, nrhs_max=2, restart_max=4, inner_k_max=2) as P:
        n = P.n
        # nvec = 0 is a no-op
        e = torch.empty(0, dtype=torch.complex128, device=DEV)
        assert P.apply_shifted(e).numel() == 0
        # zero right-hand side: u = 0, converged
        u, st = P.solve(torch.zeros(1, n, dtype=torch.complex128, device=DEV), restart=4,
                        inner_k=2)
        assert st[0].converged and float(u.abs().max()) == 0.0 and st[0].its == 0
        # invalid arguments raise, no CPU fallback
        f = torch.zeros(3, n, dtype=torch.complex128, device=DEV)
        with pytest.raises(hzpkg.HzError):
            P.shifted_solve(0, f)                                   # nvec > nrhs_max
        with pytest.raises(hzpkg.HzError):
            P.shifted_solve(5, f[:1])                               # node out of range
        with pytest.raises(hzpkg.HzError):
            P.fci(f[:1], inner_k=3)                                 # inner_k > max
        with pytest.raises(hzpkg.HzError):
            P.solve(f[:1], restart=5)                               # restart > max
        with pytest.raises(ValueError):
            P.apply_shifted(f.cpu())                                # host tensor


def test_autotuned_tiles_give_identical_results():
    """Tile shapes only change launch geometry: a problem with autotuning and one with the
    fixed defaults give bit-identical complex64 stencils and FCI outputs."""
    wl = W.small_case(14, 45, 13, 11, layer=2, J=5)
    x = W.random_field(3, 2, wl.nx, wl.ny, wl.nz)
    outs = []
    for tune in (True, False):
        P = hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t,
                          wl.eps, nrhs_max=2, restart_max=4, inner_k_max=3, autotune=tune)
        with P:
            info = P.info
            assert all(z in (1, 2, 4) for z in info["tile_poly_zc"])
            assert all(r in (1, 2, 4) for r in info["tile_poly_rows"])
            assert info["tile_stencil"][0] in (2, 4, 8) and info["tile_stencil"][1] in (2, 4, 8)
            y = to_np(P.apply_shifted(to_dev(x, torch.complex64), 0.2 - 0.7j))
            z = to_np(P.fci(to_dev(x), inner_k=3, precision=hzpkg.HZ_MIXED_C64_FCI32))
            outs.append((y, z))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_failure_statuses():
    """Non-convergence, divergence and a happy breakdown are reported, not hidden.  All are
    made on the host side: a capped cycle count, a NaN planted in the right-hand side, and an
    eigenvector right-hand side that FCI inverts exactly."""
    wl = W.small_case(4, 9, 8, 7, layer=1, J=3)
    with problem_of(wl, None, nrhs_max=1, restart_max=3, inner_k_max=2) as P:
        f = to_dev(wl.f)
        # max_cycles = 1 with an unreachable tolerance: HZ_ERR_NOT_CONVERGED, stats filled
        with pytest.raises(hzpkg.HzError) as ei:
            P.solve(f, restart=3, inner_k=2, rtol=1e-14, max_cycles=1)
        assert ei.value.status == 4
        u, st = P.solve(f, restart=3, inner_k=2, rtol=1e-14, max_cycles=1, check=False)
        assert st[0].cycles == 1 and st[0].its == 3 and not st[0].converged
        assert 0 < st[0].rel_res_true < 1
        # a NaN in the right-hand side: HZ_ERR_DIVERGED
        bad = f.clone()
        bad.view(-1)[5] = complex(float("nan"), 0.0)
        with pytest.raises(hzpkg.HzError) as ei:
            P.solve(bad, restart=3, inner_k=2, rtol=1e-8, max_cycles=3)
        assert ei.value.status == 6
        # the problem stays usable
        u, st = P.solve(f, restart=3, inner_k=2, rtol=1e-6, max_cycles=50)
        assert st[0].converged
    # eigenvector right-hand side, c = 1, no sponge: FCI returns v/mu, the first outer step
    # breaks down happily and the solve ends exactly after one step
    nx, ny, nz = 6, 5, 7
    h = 1.0 / 8
    c = np.ones((nz, ny, nx))
    omega = 2 * math.pi / (6 * h)
    with hzpkg.Problem(c, h, omega, 0, 0.0, 4, 1.0, 0.5, nrhs_max=1, restart_max=5,
                       inner_k_max=3) as P:
        i, j, k = np.arange(1, nx + 1), np.arange(1, ny + 1), np.arange(1, nz + 1)
        v = (np.sin(2 * np.pi * k / (nz + 1))[:, None, None]
             * np.sin(1 * np.pi * j / (ny + 1))[None, :, None]
             * np.sin(3 * np.pi * i / (nx + 1))[None, None, :]).astype(np.complex128)
        u, st = P.solve(to_dev(v[None]), restart=5, inner_k=3, rtol=1e-10, max_cycles=3)
        assert st[0].converged and st[0].its == 1 and st[0].rel_res_true <= 1e-12


def test_barrier_timeout_status_and_recovery():
    """A grid barrier that gives up is reported as HZ_ERR_TIMEOUT, and the problem recovers.
    The wait is made to run out on purpose by a poll limit of 0 (every barrier wait that is
    not already satisfied gives up at once: the kernel returns, nothing hangs); the next solve
    with the default limit must reproduce the first solve bit for bit."""
    wl = W.point_source_32()
    with problem_of(wl, None, nrhs_max=1, restart_max=wl.restart, inner_k_max=wl.k_in) as P:
        f = to_dev(wl.f)
        kw = dict(restart=wl.restart, inner_k=wl.k_in, rtol=1e-8, max_cycles=10,
                  precision=hzpkg.HZ_MIXED_C64_FF)
        u0, st0 = P.solve(f, **kw)
        assert st0[0].converged
        u0 = to_np(u0)
        P.set_spin_limit(0)
        with pytest.raises(hzpkg.HzError) as ei:
            P.solve(f, **kw)
        assert ei.value.status == 8, ei.value
        P.set_spin_limit(-1)
        u1, st1 = P.solve(f, **kw)
        assert st1[0].converged and st1[0].its == st0[0].its
        assert np.array_equal(to_np(u1), u0)
        # the same through the float64 cooperative kernels of the float64-outer form
        kw64 = dict(kw, precision=hzpkg.HZ_MIXED_C64)
        u2, st2 = P.solve(f, **kw64)
        P.set_spin_limit(0)
        with pytest.raises(hzpkg.HzError) as ei:
            P.solve(f, **kw64)
        assert ei.value.status == 8, ei.value
        P.set_spin_limit(-1)
        u3, st3 = P.solve(f, **kw64)
        assert st3[0].converged and np.array_equal(to_np(u3), to_np(u2))


@pytest.mark.parametrize("prec", [hzpkg.HZ_C128, hzpkg.HZ_MIXED_C64])
def test_float64_cooperative_steps_match_multi_kernel_form(prec):
    """The float64 cooperative outer Arnoldi step and FCI tail (one right-hand side) against
    the multi-kernel float64 form at a fixed step count across a restart (32^3): the same
    float64 arithmetic per point, only the grouping of the global sums differs, so the iterates
    agree to a few rounding errors amplified by the iteration (1e-10 relative)."""
    wl = W.point_source_32()
    f = to_dev(wl.f)
    kw = dict(restart=12, inner_k=4, rtol=1e-8, max_cycles=5, precision=prec, fixed_its=20)
    with problem_of(wl, None, nrhs_max=1, restart_max=12, inner_k_max=4) as P:
        u_fused, st_f = P.solve(f, **kw)
        P.fused_tail(0)
        P.fused_arnoldi(0)
        u_multi, st_m = P.solve(f, **kw)
        P.fused_tail(2)  # the summed last norm instead of the Pythagorean difference
        P.fused_arnoldi(2)
        u_sum, _ = P.solve(f, **kw)
    assert st_f[0].its == st_m[0].its == 20
    assert rel(to_np(u_fused), to_np(u_multi)) <= 1e-10
    assert rel(to_np(u_sum), to_np(u_multi)) <= 1e-10


@pytest.mark.parametrize("prec", [hzpkg.HZ_C128, hzpkg.HZ_MIXED_C64])
def test_float64_forms_converge_alike_at_64(prec):
    """At 64^3 (where the solver picks the multi-kernel float64 steps by default) the iterates
    at a fixed step count are ill-conditioned functions of the rounding (every variant differs
    from the oracle's 20-step iterate by about 4e-5 while a single FCI application agrees to
    1e-11), so the default and the modes-0 forms are compared on their converged solutions:
    both at a true residual of 1e-11, they agree to 5e-11."""
    wl = W.gaussian_bumps_64()
    f = to_dev(wl.f)
    kw = dict(restart=wl.restart, inner_k=4, rtol=1e-11, max_cycles=40, precision=prec)
    with problem_of(wl, None, nrhs_max=1, restart_max=wl.restart, inner_k_max=4) as P:
        u_fused, st_f = P.solve(f, **kw)
        P.fused_tail(0)
        P.fused_arnoldi(0)
        u_multi, st_m = P.solve(f, **kw)
    assert st_f[0].converged and st_m[0].converged
    assert rel(to_np(u_fused), to_np(u_multi)) <= 5e-11


def test_limit_flags_restrict_forms_and_keep_results():
    """HZ_LIMIT_SWEEPS_C64 refuses float64 sweeps; HZ_LIMIT_Z_C64 refuses the forms whose
    directions must stay float64 or float pairs; both problems solve the mixed form to 1e-8."""
    wl = W.point_source_32()
    fl = hzpkg.HZ_LIMIT_SWEEPS_C64 | hzpkg.HZ_LIMIT_Z_C64
    P = hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                      nrhs_max=2, restart_max=wl.restart, inner_k_max=wl.k_in, flags=fl)
    with P:
        f = to_dev(np.concatenate([wl.f, wl.f[:, ::-1]]).reshape(2, -1))
        for prec in (hzpkg.HZ_C128, hzpkg.HZ_MIXED_C64_FF):
            with pytest.raises(hzpkg.HzError) as ei:
                P.solve(f, precision=prec)
            assert ei.value.status == 1
        with pytest.raises(hzpkg.HzError) as ei:
            P.fci(f, inner_k=2, precision=hzpkg.HZ_C128)
        assert ei.value.status == 1
        for prec in (hzpkg.HZ_MIXED_C64, hzpkg.HZ_MIXED_C64_FCI32):
            u, st = P.solve(f, restart=wl.restart, inner_k=wl.k_in, rtol=1e-8, max_cycles=10,
                            precision=prec)
            assert all(s.converged for s in st)
            op, _ = oracle_of(wl)
            for r in range(2):
                fr = to_np(f)[r].reshape(op.shape) * op.s
                ur = to_np(u)[r].reshape(op.shape)
                assert np.linalg.norm(fr - op.apply(ur)) / np.linalg.norm(fr) <= 1e-8


def test_native_kernels_launch():
    before = hzpkg.launch_count()
    wl = W.small_case(1, 8, 8, 8, layer=1, J=2)
    with problem_of(wl) as P:
        P.apply_shifted(torch.ones(1, P.n, dtype=torch.complex128, device=DEV))
        torch.cuda.synchronize()
    assert hzpkg.launch_count() > before


# ---------------------------------------------------------------------------------- Case Two
def case_two_problem(wl, nrhs_max=1, restart_max=10, inner_k_max=3):
    return hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                         nrhs_max=nrhs_max, restart_max=restart_max, inner_k_max=inner_k_max,
                         flags=hzpkg.HZ_LIMIT_CASE_TWO)


@pytest.mark.parametrize("shape,layer", [((13, 9, 7), 2), ((32, 32, 32), 8)])
def test_case_two_nodes_and_fci_match_oracle(shape, layer):
    """Case Two (eq:mat-2x2): the contour and polynomial parameters from the rectangle of the
    Remark after Theorem thm:spectrum-2x2 equal the oracle's setup_nodes_2x2, and FCI on iC - I
    (Algorithm 1 with the scheme eq:fix-pt-exp on the 2n-point fields) equals the oracle's on
    the same input: 1e-11 relative (float64)."""
    wl = W.small_case(11, *shape, layer=layer, J=4) if shape[0] != 32 else W.point_source_32()
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    _, nodes = O.setup_nodes_2x2(op, wl.J, wl.t, wl.eps)
    with case_two_problem(wl, nrhs_max=2, inner_k_max=4) as P:
        tb = P.nodes()
        assert list(tb["q"]) == [nd.q for nd in nodes]
        assert list(tb["sweeps"]) == [nd.sweeps for nd in nodes]
        assert np.allclose(tb["z"], [nd.z for nd in nodes], rtol=1e-12, atol=1e-14)
        assert np.allclose(tb["delta"], [nd.delta for nd in nodes], rtol=1e-7)
        r = W.random_field(13, 2, wl.nx, wl.ny, 2 * wl.nz)  # two stacked fields per vector
        out = to_np(P.fci(to_dev(r.reshape(2, -1)), inner_k=4)).reshape(2, -1)
    op2 = O.Operator2x2(op)
    for v in range(2):
        ref = O.fci(op2, r[v].reshape(op2.shape), nodes, 4)
        assert rel(out[v], ref) <= 1e-11


def test_case_two_solve_fixed_steps_match_oracle():
    """FGMRES(5) with FCI on iC - I across two restarts equals the oracle's solve_2x2 at a
    fixed step count (iterates Y, float64)."""
    wl = W.small_case(3, 13, 9, 7, layer=2, J=4)
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    _, nodes = O.setup_nodes_2x2(op, wl.J, wl.t, wl.eps)
    res = O.solve_2x2(op, op.s * wl.f[0], nodes, m=5, k_in=3, rtol=1e-30, max_cycles=100,
                      fixed_its=12)
    with case_two_problem(wl, restart_max=5) as P:
        Y, st = P.solve(to_dev(wl.f.reshape(1, -1)), restart=5, inner_k=3, rtol=1e-30,
                        max_cycles=100, fixed_its=12)
    assert st[0].its == 12 and st[0].cycles == res.cycles
    assert rel(to_np(Y)[0], res.u) <= 1e-9
    assert st[0].rel_res_true == pytest.approx(res.rel_res_true, rel=1e-6)


def test_case_two_solves_point_source_32():
    """Case Two on the 32^3 point source to 1e-8: the 2x2 residual of the returned Y, from the
    oracle's Operator2x2, equals the reported one; Y's halves satisfy Y1 = i Y2 and Case One's
    residual of u = Y2 is reported (it is bounded by the 2x2 residual times the coupling)."""
    wl = W.point_source_32()
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    op2 = O.Operator2x2(op)
    with case_two_problem(wl, restart_max=wl.restart, inner_k_max=wl.k_in) as P:
        Y, st = P.solve(to_dev(wl.f.reshape(1, -1)), restart=wl.restart, inner_k=wl.k_in,
                        rtol=1e-8, max_cycles=40)
    assert st[0].converged
    Yn = to_np(Y)[0].reshape(op2.shape)
    F = np.stack([np.zeros(op.shape, dtype=np.complex128), op.s * wl.f[0]])
    res2 = np.linalg.norm(F - op2.apply(Yn)) / np.linalg.norm(F)
    assert res2 <= 1e-8 + 1e-12 and abs(res2 - st[0].rel_res_true) <= 1e-10
    res1 = np.linalg.norm(op.s * wl.f[0] - op.apply(Yn[1])) / np.linalg.norm(op.s * wl.f[0])
    print(f"Case Two 32^3: {st[0].its} steps, 2x2 residual {res2:.2e}, Case One residual of "
          f"u = Y2 {res1:.2e}")
    assert res1 <= 1e-6


# ---------------------------------------------------------------------- ILU(0) (§6.3, §7.3)
@pytest.mark.parametrize("shape,layer", [((37, 19, 11), 3), ((1, 1, 1), 0), ((32, 32, 32), 8),
                                         ((20, 24, 37), 2), ((40, 64, 50), 4)],
                         ids=lambda v: str(v))
def test_ilu0_apply_matches_oracle(shape, layer):
    """z = M^{-1} t with the ILU(0) factors of the 7-point Laplacian: the GPU's hyperplane sweeps
    against the oracle's (two right-hand sides, ragged and degenerate grids): 1e-13.  The last
    three grids run the multi-block wavefront (z-slabs of 512 / ny planes: 2 slabs at 32^3, 2
    ragged at 24 x 37, 7 ragged at 64 x 50), the first two the one-block sweeps."""
    wl = W.small_case(21, *shape, layer=layer, J=2)
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    Minv = O.ilu0_preconditioner(op)
    t = W.random_field(22, 2, wl.nx, wl.ny, wl.nz)
    with problem_of(wl, None, nrhs_max=2) as P:
        P.set_inner_ilu(True)
        z = to_np(P.ilu0_apply(to_dev(t.reshape(2, -1))))
    for v in range(2):
        assert rel(z[v], Minv(t[v])) <= 1e-13


@pytest.mark.parametrize("shape", [(13, 9, 7), (24, 32, 20)], ids=str)
@pytest.mark.parametrize("prec,tol", [(hzpkg.HZ_C128, 1e-11), (hzpkg.HZ_MIXED_C64, 1e-5)])
def test_fci_with_ilu0_inner_preconditioner_matches_oracle(prec, tol, shape):
    """Algorithm 1 with the inner GMRES right-preconditioned by ILU(0) (one and two right-hand
    sides per call) against the oracle's fci(..., inner_precond).  The mixed form takes its
    complex64 polynomial sweeps and float32 ILU(0) sweeps (1e-5, as for its FCI without ILU);
    the all-float64 form its float64 ones (1e-11).  13 x 9 x 7 runs the one-block sweeps,
    24 x 32 x 20 the multi-block wavefront (two z-slabs, the second ragged)."""
    wl = W.small_case(3, *shape, layer=2, J=4)
    op, nodes = oracle_of(wl)
    Minv = O.ilu0_preconditioner(op)
    r = W.random_field(5, 2, wl.nx, wl.ny, wl.nz)
    with problem_of(wl, nodes, nrhs_max=2, inner_k_max=4) as P:
        P.set_inner_ilu(True)
        out = to_np(P.fci(to_dev(r.reshape(2, -1)), inner_k=3, precision=prec))
        out1 = to_np(P.fci(to_dev(r[:1].reshape(1, -1)), inner_k=3, precision=prec))
        with pytest.raises(hzpkg.HzError):
            P.fci(to_dev(r[:1].reshape(1, -1)), inner_k=3, precision=hzpkg.HZ_MIXED_C64_FCI32)
    for v in range(2):
        ref = O.fci(op, r[v], nodes, 3, inner_precond=Minv)
        assert rel(out[v], ref) <= tol
    assert rel(out1[0], O.fci(op, r[0], nodes, 3, inner_precond=Minv)) <= tol


def test_solve_with_ilu0_converges_and_reports_steps():
    """FGMRES with FCI whose inner GMRES is ILU(0)-preconditioned reaches the float64 true
    residual 1e-8 on the 32^3 point source; iterates at a fixed step count equal the oracle's
    solve with the same inner preconditioner (1e-9, small grid)."""
    wl = W.small_case(3, 13, 9, 7, layer=2, J=4)
    op, nodes = oracle_of(wl)
    Minv = O.ilu0_preconditioner(op)
    res = O.solve(op, op.s * wl.f[0], nodes, m=5, k_in=3, rtol=1e-30, max_cycles=100,
                  fixed_its=12, inner_precond=Minv)
    with problem_of(wl, nodes, nrhs_max=1, restart_max=5, inner_k_max=3) as P:
        P.set_inner_ilu(True)
        u, st = P.solve(to_dev(wl.f), restart=5, inner_k=3, rtol=1e-30, max_cycles=100,
                        fixed_its=12)
    assert rel(to_np(u)[0], res.u) <= 1e-9
    wl = W.point_source_32()
    with problem_of(wl, None, nrhs_max=1, restart_max=wl.restart, inner_k_max=wl.k_in) as P:
        f = to_dev(wl.f)
        kw = dict(restart=wl.restart, inner_k=wl.k_in, rtol=1e-8, max_cycles=40,
                  precision=hzpkg.HZ_MIXED_C64)
        _, st0 = P.solve(f, **kw)
        P.set_inner_ilu(True)
        u, st1 = P.solve(f, **kw)
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    sf = op.s * wl.f[0]
    assert st1[0].converged
    assert np.linalg.norm(sf - op.apply(to_np(u)[0].reshape(op.shape))) / np.linalg.norm(sf) <= 1e-8 + 1e-12
    print(f"32^3 outer steps to 1e-8: FCI {st0[0].its}, FCI with ILU(0) inner GMRES {st1[0].its}")
