"""GPU parity of the Fourier spectral discretisation (Section 7.1 eq:eig-Laplacian-spectral) and
of the regularised inverse-Laplacian inner preconditioner (Section 7.3) against the oracle.

Grids: powers of two, products of 2, 3 and 5 with ragged tiles, a line of length 1, and 64^3.
Tolerances (relative L2): float64 operator 1e-13 (line FFTs of up to 64 points: a few hundred
roundings of 1e-16 relative to the largest mode), float64 polynomial solve 1e-12, float64
FCI 1e-11, complex64 operator 1e-5 and complex64 sweeps / mixed FCI 1e-5 (float32 FFT
rounding, about log2(n) eps_32 relative to the field's largest mode, through contracting
iterations); full solves to rtol 1e-11 against the oracle's 1e-12 solution within 1e-9 (float64)
and the outer tolerance 1e-8 (mixed).
"""
import numpy as np
import pytest

import workloads as W
from oracle import hz_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1811_12378_gb300 as hzpkg  # noqa: E402

DEV = "cuda:0"
SPEC = hzpkg.HZ_DISC_SPECTRAL


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV).to(dtype).contiguous()


def to_np(t):
    return t.detach().cpu().numpy()


def spectral_oracle(wl, t=None):
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, kind="spectral")
    (_, _, _), nodes = O.setup_nodes(op, wl.J, wl.t if t is None else t, wl.eps)
    return op, nodes


def spectral_problem(wl, nodes=None, nrhs_max=2, restart_max=30, inner_k_max=6, t=None,
                     flags=0):
    P = hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J,
                      wl.t if t is None else t, wl.eps, nrhs_max=nrhs_max,
                      restart_max=restart_max, inner_k_max=inner_k_max, flags=flags,
                      discretization=SPEC)
    if nodes is not None:
        P.set_nodes([nd.z for nd in nodes], [nd.sigma for nd in nodes], [nd.z0 for nd in nodes],
                    [nd.delta for nd in nodes], [nd.q for nd in nodes],
                    [nd.sweeps for nd in nodes])
    return P


# lines of 32-256 points take the compiled sizes; the last four have 64- and 256-point y and z
# lines (the complex64 register-staged tiles of 32 and 16 x positions) under x extents that
# leave the tiles ragged
GRIDS = [((16, 16, 16), 2), ((30, 12, 10), 2), ((1, 8, 6), 1), ((25, 9, 20), 3),
         ((64, 64, 64), 8), ((128, 32, 12), 2), ((256, 10, 32), 2), ((12, 256, 10), 2),
         ((20, 8, 256), 2), ((20, 64, 12), 2), ((40, 12, 64), 2)]


@pytest.mark.parametrize("shape,layer", GRIDS, ids=lambda v: str(v))
def test_spectral_operator_matches_oracle(shape, layer):
    """(A - zI) x with the spectral Laplacian, three fields per call, float64 and complex64."""
    wl = W.small_case(4, *shape, layer=layer, ppw=3.0, J=2)
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, kind="spectral")
    x = W.random_field(5, 3, wl.nx, wl.ny, wl.nz)
    z = 0.37 - 0.81j
    with spectral_problem(wl) as P:
        y = to_np(P.apply_shifted(to_dev(x.reshape(3, -1)), z))
        y32 = to_np(P.apply_shifted(to_dev(x.reshape(3, -1), torch.complex64), z,
                                    precision=hzpkg.HZ_MIXED_C64))
    for v in range(3):
        ref = op.apply(x[v], z)
        assert rel(y[v], ref) <= 1e-13
        assert rel(y32[v], ref) <= 1e-5


@pytest.mark.parametrize("shape", [(16, 16, 16), (30, 12, 10), (1, 8, 6)], ids=str)
def test_inverse_laplacian_matches_oracle(shape):
    """z = F^H diag(1/max(lambda, 1)) F t against the oracle (two fields; in place too)."""
    wl = W.small_case(6, *shape, layer=1, ppw=3.0, J=2)
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, kind="spectral")
    Minv = O.invlap_preconditioner(op)
    t = W.random_field(7, 2, wl.nx, wl.ny, wl.nz)
    with spectral_problem(wl) as P:
        z = to_np(P.invlap_apply(to_dev(t.reshape(2, -1))))
        tt = to_dev(t.reshape(2, -1))
        P.invlap_apply(tt, out=tt)
        z2 = to_np(tt)
    for v in range(2):
        assert rel(z[v], Minv(t[v])) <= 1e-13
        assert rel(z2[v], Minv(t[v])) <= 1e-13


@pytest.mark.parametrize("shape", [(16, 16, 16), (30, 12, 10)], ids=str)
def test_spectral_shifted_solve_matches_oracle(shape):
    """The polynomial scheme (eq:fix-pt-exp) at every node on the spectral operator: float64
    1e-12, complex64 sweeps 1e-5."""
    wl = W.small_case(8, *shape, layer=2, ppw=3.0, J=4)
    op, nodes = spectral_oracle(wl)
    f = W.random_field(9, 2, wl.nx, wl.ny, wl.nz)
    with spectral_problem(wl, nodes) as P:
        for j, nd in enumerate(nodes):
            y = to_np(P.shifted_solve(j, to_dev(f.reshape(2, -1))))
            y32 = to_np(P.shifted_solve(j, to_dev(f.reshape(2, -1), torch.complex64),
                                        precision=hzpkg.HZ_MIXED_C64))
            for v in range(2):
                ref = O.poly_solve(op, f[v], nd)
                assert rel(y[v], ref) <= 1e-12
                assert rel(y32[v], ref) <= 1e-5


@pytest.mark.parametrize("invlap", [False, True])
@pytest.mark.parametrize("kin", [0, 3])
def test_spectral_fci_matches_oracle(invlap, kin):
    """Algorithm 1 on the spectral operator (two right-hand sides), with and without the
    inverse-Laplacian inner preconditioner: float64 1e-11, mixed form 1e-5."""
    wl = W.small_case(10, 20, 18, 16, layer=2, ppw=2.5, J=6)
    op, nodes = spectral_oracle(wl)
    pre = O.invlap_preconditioner(op) if invlap else None
    r = W.random_field(11, 2, wl.nx, wl.ny, wl.nz)
    with spectral_problem(wl, nodes) as P:
        P.set_inner_invlap(invlap)
        out = to_np(P.fci(to_dev(r.reshape(2, -1)), inner_k=kin, precision=hzpkg.HZ_C128))
        out32 = to_np(P.fci(to_dev(r.reshape(2, -1)), inner_k=kin,
                            precision=hzpkg.HZ_MIXED_C64))
        with pytest.raises(hzpkg.HzError):
            P.fci(to_dev(r[:1].reshape(1, -1)), inner_k=kin,
                  precision=hzpkg.HZ_MIXED_C64_FCI32)
    for v in range(2):
        ref = O.fci(op, r[v], nodes, kin, inner_precond=pre)
        assert rel(out[v], ref) <= 1e-11
        assert rel(out32[v], ref) <= 1e-5


@pytest.mark.parametrize("invlap", [False, True])
def test_spectral_solve_error_vs_oracle(invlap):
    """FGMRES + FCI on the spectral workload (24^3 periodic box, 2.25 points per wavelength in
    the background) on an ellipse contour t = 0.6 (Section 6.1): solved to a true residual of
    1e-11 on both sides, the GPU solution is within 1e-9 (HZ_C128) and 1e-8 (HZ_MIXED_C64) of
    the oracle's; at rtol 1e-8 the step counts agree within 2."""
    wl = W.spectral_bumps(24, 3)
    op, nodes = spectral_oracle(wl, t=0.6)
    pre = O.invlap_preconditioner(op) if invlap else None
    f = wl.f[0]  # physical units: the library solves A u = s f, the oracle takes s f
    ref = O.solve(op, op.s * f, nodes, m=30, k_in=4, rtol=1e-12, max_cycles=40,
                  inner_precond=pre)
    ref8 = O.solve(op, op.s * f, nodes, m=30, k_in=4, rtol=1e-8, max_cycles=40,
                   inner_precond=pre)
    assert ref.converged and ref8.converged
    with spectral_problem(wl, nodes, nrhs_max=1, inner_k_max=4, t=0.6) as P:
        P.set_inner_invlap(invlap)
        fd = to_dev(f.reshape(1, -1))
        for prec, tol in ((hzpkg.HZ_C128, 1e-9), (hzpkg.HZ_MIXED_C64, 1e-8)):
            u, st = P.solve(fd, restart=30, inner_k=4, rtol=1e-11, max_cycles=40, precision=prec)
            assert st[0].converged and st[0].rel_res_true <= 1e-11
            assert rel(to_np(u)[0], ref.u) <= tol
            u8, st8 = P.solve(fd, restart=30, inner_k=4, rtol=1e-8, max_cycles=40,
                              precision=prec)
            assert st8[0].converged and st8[0].rel_res_true <= 1e-8
            assert abs(st8[0].its - ref8.its) <= 2


def test_spectral_multi_rhs_and_batched_solves():
    """Two right-hand sides in one spectral solve equal two single solves (HZ_MIXED_C64, bit for
    bit: the batched kernels keep every field's arithmetic), and hz_solve_batched runs a
    spectral and a 7-point problem together with the results of separate solves."""
    wl = W.spectral_bumps(24, 5)
    op, nodes = spectral_oracle(wl)
    f2 = np.stack([wl.f[0], W.random_field(3, 1, wl.nx, wl.ny, wl.nz)[0]]).reshape(2, -1)
    kw = dict(restart=20, inner_k=4, rtol=1e-8, max_cycles=40, precision=hzpkg.HZ_MIXED_C64)
    with spectral_problem(wl, nodes, nrhs_max=2, inner_k_max=4) as P:
        u2, st2 = P.solve(to_dev(f2), **kw)
        u2 = to_np(u2)
        for v in range(2):
            u1, st1 = P.solve(to_dev(f2[v:v + 1]), **kw)
            assert st1[0].its == st2[v].its and st2[v].converged
            assert np.array_equal(to_np(u1)[0], u2[v])
        wf = W.small_case(4, 20, 16, 12, layer=2, J=4)
        with hzpkg.Problem(wf.c, wf.h, wf.omega, wf.layer_cells, wf.sigma_max, wf.J, wf.t,
                           wf.eps, nrhs_max=1, restart_max=20, inner_k_max=4) as Q:
            fq = to_dev(wf.f[:1].reshape(1, -1))
            # a batch runs the per-piece Krylov kernels; the lone solve of one right-hand side
            # would otherwise take the cooperative ones (other rounding)
            Q.fused_tail(0)
            Q.fused_arnoldi(0)
            us, sts = hzpkg.solve_batched([P, Q], [to_dev(f2[:1]), fq], **kw)
            uq, stq = Q.solve(fq, **kw)
            assert np.array_equal(to_np(us[0])[0], u2[0]) and sts[0][0].its == st2[0].its
            assert np.array_equal(to_np(us[1]), to_np(uq)) and sts[1][0].its == stq[0].its
    sf = op.s * f2[0].reshape(op.shape)
    assert np.linalg.norm(sf - op.apply(u2[0].reshape(op.shape))) / np.linalg.norm(sf) <= 1.01e-8


def test_spectral_argument_checks():
    """Sizes outside 2^a 3^b 5^c, Case Two, the complex64-Krylov forms, ILU(0) and the network
    are refused on a spectral problem; the inverse Laplacian on a 7-point one."""
    wl = W.small_case(2, 14, 8, 8, layer=1, ppw=3.0, J=2)
    with pytest.raises(hzpkg.HzError):
        spectral_problem(wl)  # 14 = 2 x 7
    wl = W.small_case(2, 12, 8, 8, layer=1, ppw=3.0, J=2)
    with pytest.raises(hzpkg.HzError):
        spectral_problem(wl, flags=hzpkg.HZ_LIMIT_CASE_TWO)
    with spectral_problem(wl) as P:
        with pytest.raises(hzpkg.HzError):
            P.set_inner_ilu(True)
        f = to_dev(W.random_field(1, 1, wl.nx, wl.ny, wl.nz).reshape(1, -1))
        with pytest.raises(hzpkg.HzError):
            P.solve(f, restart=5, inner_k=2, precision=hzpkg.HZ_MIXED_C64_FF)
    with hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t,
                       wl.eps) as Q:
        with pytest.raises(hzpkg.HzError):
            Q.set_inner_invlap(True)
