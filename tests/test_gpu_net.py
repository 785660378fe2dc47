"""The learned preconditioner's tensor-core kernels and network against the CPU oracle
(oracle/hz_net_oracle.py), and its use as a right preconditioner in FGMRES.

Tolerances.  A single convolution takes bf16 operands and accumulates in fp32 on the tensor
cores; the oracle sums the same bf16 values in float64, so the difference is fp32 rounding of
sums of up to 27 * 192 products: relative L2 <= 1e-5, each element within 1e-4 of the output's
largest magnitude.  The weight gradient sums up to 16^3 * 2 products per entry, split over
blocks and added with float atomics: relative L2 <= 1e-4.  The whole network stores every
feature map in bf16; the oracle's bf16 mode rounds at the same points, so the remaining
difference is fp32-versus-float64 summation that moves some values across a bf16 rounding
boundary: a sum of K products carries an fp32 error of about sqrt(K) 2^-24 relative, against
a bf16 spacing of 2^-8, so about sqrt(K) 2^-16 (0.1% at K = 27 * 192) of each layer's stored
values flip by one bf16 ulp (2^-8 relative), and the flips compound over the network's ~30
rounding points.  Bounds: relative L2 <= 5e-3 for the output; for the gradients <= 1e-2 over
all parameters together and <= 5e-2 for each parameter tensor (the bottleneck's weight
gradient sums over only D^3/512 voxels per sample at the end of nine rounded backward levels,
so a few flipped values move it by percents; a structural mistake -- a wrong tap, transposed
channels, a dropped skip path -- gives errors of order one).
"""
import numpy as np
import pytest

import workloads as W
from oracle import hz_net_oracle as N
from oracle import hz_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1811_12378_gb300 as hzpkg  # noqa: E402

DEV = "cuda:0"


def rng(s):
    return np.random.Generator(np.random.PCG64(s))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def bf16_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV).to(torch.bfloat16)


CONV_CASES = [  # (B, D, H, W, Cin, Cout, relu)
    (1, 16, 16, 16, 16, 16, False),   # the 16^3 x 16-channel case
    (2, 8, 16, 32, 8, 16, True),      # 27 chunks (odd: a padded MMA), batch of two, ReLU
    (1, 8, 8, 8, 48, 16, False),      # concatenated-width input, 8^3 (one tile)
    (1, 16, 8, 24, 16, 128, True),    # wide output, ragged x (24 = not a multiple of 32)
    (1, 8, 8, 8, 128, 64, False),     # deep input
]


@pytest.mark.parametrize("B,D,H,W,cin,cout,relu", CONV_CASES)
def test_conv3d_forward_matches_oracle(B, D, H, W, cin, cout, relu):
    g = rng(10 + cin + cout)
    x = N.bf16_round(g.standard_normal((B, D, H, W, cin)).astype(np.float32))
    w = (g.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin)).astype(np.float32)
    b = g.standard_normal(cout).astype(np.float32)
    y = hzpkg.conv3d(bf16_dev(x), torch.from_numpy(w).to(DEV), torch.from_numpy(b).to(DEV),
                     relu=relu).cpu().numpy()
    wq = N.bf16_round(w)
    for s in range(B):
        ref = N.conv3(x[s], wq, b)
        if relu:
            ref = N.relu(ref)
        assert rel(y[s], ref) <= 1e-5
        assert np.max(np.abs(y[s] - ref)) <= 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("B,D,H,W,cin,cout", [(1, 16, 16, 16, 16, 16), (2, 8, 8, 16, 32, 64),
                                              (1, 8, 16, 8, 64, 128)])
def test_conv3d_backward_matches_oracle(B, D, H, W, cin, cout):
    g = rng(20 + cin)
    x = N.bf16_round(g.standard_normal((B, D, H, W, cin)).astype(np.float32))
    gr = N.bf16_round(g.standard_normal((B, D, H, W, cout)).astype(np.float32))
    w = (g.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin)).astype(np.float32)
    dx, dw = hzpkg.conv3d_backward(bf16_dev(x), bf16_dev(gr), torch.from_numpy(w).to(DEV))
    dx, dw = dx.cpu().numpy(), dw.cpu().numpy()
    wq = N.bf16_round(w)
    dw_ref = np.zeros_like(dw, dtype=np.float64)
    for s in range(B):
        dxs, dws, _ = N.conv3_backward(x[s], wq, gr[s])
        dw_ref += dws
        assert rel(dx[s], dxs) <= 1e-5
    assert rel(dw, dw_ref) <= 1e-4


def _net_case(seed, B, D):
    g = rng(seed)
    p = N.init_params(seed)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * g.standard_normal(p[k].shape)
    x = g.standard_normal((B, D, D, D, 8)).astype(np.float32)
    x[..., 3:] = 0.0
    t = g.standard_normal((B, D, D, D, 2)).astype(np.float32)
    return p, x, t


@pytest.mark.parametrize("B,D", [(1, 8), (2, 16)])
def test_network_forward_and_gradients_match_oracle(B, D):
    p, x, t = _net_case(31 + D, B, D)
    with hzpkg.Net(D, D, D, batch_max=B) as net:
        net.set_params(hzpkg.flatten_params(p))
        xd = torch.from_numpy(x).to(DEV)
        y = net.forward(xd).cpu().numpy()
        loss, gflat = net.train_step(xd, torch.from_numpy(t).to(DEV), lr=0.0, want_grads=True)
        grads = hzpkg.unflatten_params(gflat.cpu().numpy())
        # lr = 0 leaves the parameters untouched
        assert np.array_equal(net.get_params(), hzpkg.flatten_params(p))
    ref_loss = 0.0
    ref_g = {k: 0.0 for k in p}
    yerr = []
    for s in range(B):
        ys, cache = N.forward(p, x[s].astype(np.float64), keep=True, bf16=True)
        yerr.append(rel(y[s], ys))
        assert yerr[-1] <= 5e-3, yerr
        ls, dy = N.loss_mse(ys, t[s])
        ref_loss += ls
        gs = N.backward(p, cache, dy)
        for k in p:
            ref_g[k] = ref_g[k] + gs[k]
    assert abs(loss - ref_loss) <= 5e-3 * ref_loss
    errs = {k: rel(grads[k], ref_g[k]) for k in p}
    worst = max(errs, key=errs.get)
    gall = np.concatenate([np.ravel(grads[k]) for k in p])
    rall = np.concatenate([np.ravel(ref_g[k]) for k in p])
    print(f"{B} x {D}^3: output rel. L2 vs oracle {max(yerr):.1e}; gradients: all "
          f"{rel(gall, rall):.1e}, median tensor {np.median(list(errs.values())):.1e}, worst "
          f"{worst} {errs[worst]:.1e}")
    assert rel(gall, rall) <= 1e-2
    assert errs[worst] <= 5e-2, errs


def test_training_lowers_the_loss():
    """Adam steps on a fixed batch with a learnable target (a pointwise mixing of the input's
    two field channels); the oracle's own update rule is pinned on the CPU."""
    p, x, _ = _net_case(41, 2, 16)
    t = np.stack([0.5 * (x[..., 0] + x[..., 1]), 0.5 * (x[..., 0] - x[..., 1])], axis=-1)
    with hzpkg.Net(16, 16, 16, batch_max=2) as net:
        net.set_params(hzpkg.flatten_params(p))
        xd = torch.from_numpy(x).to(DEV)
        td = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).to(DEV)
        # the first step's update equals the oracle's Adam step on the library's own gradients
        p0 = net.get_params().astype(np.float64)
        l0, g0 = net.train_step(xd, td, lr=1e-3, want_grads=True)
        ref = {"a": p0.copy()}
        N.adam_step(ref, {"a": g0.cpu().numpy().astype(np.float64)}, {}, lr=1e-3)
        p1 = net.get_params()
        assert np.max(np.abs(p1 - ref["a"])) <= 1e-6 * (1.0 + np.max(np.abs(p0)))
        losses = [l0] + [net.train_step(xd, td, lr=1e-3)[0] for _ in range(39)]
    assert losses[-1] < 0.7 * losses[0], losses


def _training_pairs(P, wl, k, seed):
    """(r, e) with A e = r: r smooth random fields, e from the library's solve (rtol 1e-8)."""
    g = rng(seed)
    n = P.n
    r = g.standard_normal((k, wl.nz, wl.ny, wl.nx)) + 1j * g.standard_normal((k, wl.nz, wl.ny, wl.nx))
    for _ in range(3):  # a few box-filter passes: broadband but not white
        r = (r + np.roll(r, 1, 1) + np.roll(r, -1, 1) + np.roll(r, 1, 2) + np.roll(r, -1, 2)
             + np.roll(r, 1, 3) + np.roll(r, -1, 3)) / 7.0
    rd = torch.from_numpy(r.reshape(k, n)).to(DEV)
    # A e = r in normalised units: the solver takes physical right-hand sides f = r / s
    s = P.info["s"]
    e, st = P.solve(rd / s, restart=wl.restart, inner_k=wl.k_in, rtol=1e-8, max_cycles=20,
                    precision=hzpkg.HZ_MIXED_C64)
    assert all(x.converged for x in st)
    return rd, e


def test_learned_preconditioner_in_fgmres():
    """Train on (residual, error) pairs of the 32^3 point-source problem, then solve with the
    network as the correction after FCI (mode 3), before FCI with its least-squares step
    (mode 2) and alone (mode 1): the float64 true residual still reaches 1e-8 (it alone decides
    convergence), the solution matches the oracle's matvec residual, mode 2 needs no more
    outer steps than FCI alone, and the step counts are reported."""
    wl = W.point_source_32()
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    P = hzpkg.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                      nrhs_max=4, restart_max=wl.restart, inner_k_max=wl.k_in)
    net = hzpkg.Net(32, 32, 32, batch_max=4)
    try:
        net.set_params(hzpkg.flatten_params(N.init_params(5)))
        r, e = _training_pairs(P, wl, 4, 77)
        losses = [net.train_fields(P, r, e, lr=1e-3) for _ in range(40)]
        assert losses[-1] < losses[0]
        f = torch.from_numpy(wl.f.reshape(1, -1).copy()).to(DEV)
        kw = dict(restart=wl.restart, inner_k=wl.k_in, rtol=1e-8, max_cycles=40,
                  precision=hzpkg.HZ_MIXED_C64)
        _, st0 = P.solve(f, **kw)
        its = {0: st0[0].its}
        P.set_preconditioner(net, 3)
        u, st = P.solve(f, **kw)
        assert st[0].converged and st[0].rel_res_true <= 1e-8
        un = u.cpu().numpy().reshape(op.shape)
        sf = op.s * wl.f[0]
        assert np.linalg.norm(sf - op.apply(un)) / np.linalg.norm(sf) <= 1e-8 + 1e-12
        its[3] = st[0].its
        # the network first with its least-squares step, FCI on the rest (mode 2): the step
        # keeps a weak network from raising the residual, so FGMRES needs no more outer steps
        # than with FCI alone (two steps of slack for the variable preconditioner)
        P.set_preconditioner(net, 2)
        u2, st2 = P.solve(f, **kw)
        assert st2[0].converged and st2[0].rel_res_true <= 1e-8
        un2 = u2.cpu().numpy().reshape(op.shape)
        assert np.linalg.norm(sf - op.apply(un2)) / np.linalg.norm(sf) <= 1e-8 + 1e-12
        its[2] = st2[0].its
        assert its[2] <= its[0] + 2
        # the network alone: a weak preconditioner after this little training; the solve runs a
        # bounded number of cycles and must report its true residual honestly
        P.set_preconditioner(net, 1)
        u1, st1 = P.solve(f, **dict(kw, max_cycles=4), check=False)
        un1 = u1.cpu().numpy().reshape(op.shape)
        assert abs(np.linalg.norm(sf - op.apply(un1)) / np.linalg.norm(sf)
                   - st1[0].rel_res_true) <= 1e-9 + 1e-6 * st1[0].rel_res_true
        its[1] = (st1[0].its, st1[0].rel_res_true)
        P.set_preconditioner(None, 0)
        print(f"outer steps to 1e-8: FCI {its[0]}, network + FCI {its[2]}, FCI + network "
              f"{its[3]}; network alone {its[1][0]} steps reach {its[1][1]:.2e}")
    finally:
        net.close()
        P.close()
