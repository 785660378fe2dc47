"""Pins of the learned preconditioner's CPU oracle (oracle/hz_net_oracle.py) against things
other than itself: a library correlation routine, an explicit patch-matrix product, finite
differences, adjoint identities, closed forms and torch's own bfloat16 rounding.  A dropped
tap, a flipped offset, a transposed weight, a missing ReLU mask or skip path fails one of them.
"""
import numpy as np
import pytest

from oracle import hz_net_oracle as N

scipy_signal = pytest.importorskip("scipy.signal")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3_matches_library_correlation():
    """Each output channel is the sum over input channels of scipy's 'same' correlation with
    the 3x3x3 kernel (zero padding), plus the bias."""
    g = rng(1)
    x = g.standard_normal((6, 5, 7, 3))
    w = g.standard_normal((2, 27, 3))
    b = g.standard_normal(2)
    out = N.conv3(x, w, b)
    for co in range(2):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            k = w[co, :, ci].reshape(3, 3, 3)  # taps t = 9 dz + 3 dy + dx
            ref += scipy_signal.correlate(x[..., ci], k, mode="same", method="direct")
        assert np.allclose(out[..., co], ref, rtol=1e-12, atol=1e-12)


def test_conv3_matches_patch_matrix_product():
    """out = patches @ w.T with patches[v, (t, ci)] = x[v + offset_t, ci] built point by point."""
    g = rng(2)
    D, H, W, C = 4, 3, 5, 2
    x = g.standard_normal((D, H, W, C))
    w = g.standard_normal((3, 27, C))
    P = np.zeros((D * H * W, 27 * C))
    for z in range(D):
        for y in range(H):
            for xx in range(W):
                v = (z * H + y) * W + xx
                for dz in range(3):
                    for dy in range(3):
                        for dx in range(3):
                            zz, yy, x3 = z + dz - 1, y + dy - 1, xx + dx - 1
                            if 0 <= zz < D and 0 <= yy < H and 0 <= x3 < W:
                                t = 9 * dz + 3 * dy + dx
                                P[v, t * C:(t + 1) * C] = x[zz, yy, x3]
    ref = P @ w.reshape(3, 27 * C).T
    assert np.allclose(N.conv3(x, w).reshape(-1, 3), ref, rtol=1e-12, atol=1e-12)


def test_conv3_backward_is_the_adjoint_and_matches_finite_differences():
    g = rng(3)
    x = g.standard_normal((4, 5, 3, 3))
    w = g.standard_normal((2, 27, 3))
    b = g.standard_normal(2)
    R = g.standard_normal((4, 5, 3, 2))
    dx, dw, db = N.conv3_backward(x, w, R)
    # <conv3(x, w), R> = <x, dx> (the input gradient is the adjoint of the linear map x -> out)
    assert np.isclose(np.sum(N.conv3(x, w) * R), np.sum(x * dx), rtol=1e-12)
    assert np.isclose(np.sum(N.conv3(x, w) * R), np.sum(w * dw), rtol=1e-12)

    def loss(xx, ww, bb):
        return float(np.sum(N.conv3(xx, ww, bb) * R))
    hstep = 1e-6
    for idx in [(0, 0, 0, 0), (3, 4, 2, 1), (2, 1, 1, 2)]:
        e = np.zeros_like(x)
        e[idx] = hstep
        fd = (loss(x + e, w, b) - loss(x - e, w, b)) / (2 * hstep)
        assert np.isclose(fd, dx[idx], rtol=1e-6, atol=1e-9)
    for idx in [(0, 0, 0), (1, 13, 2), (0, 26, 1)]:
        e = np.zeros_like(w)
        e[idx] = hstep
        fd = (loss(x, w + e, b) - loss(x, w - e, b)) / (2 * hstep)
        assert np.isclose(fd, dw[idx], rtol=1e-6, atol=1e-9)
    assert np.allclose(db, R.reshape(-1, 2).sum(0))


def test_pool_and_upsample_identities():
    g = rng(4)
    x = g.standard_normal((4, 6, 2, 3))
    y = g.standard_normal((2, 3, 1, 3))
    # up2 and its adjoint; avgpool2 = up2^T / 8; pooling a constant keeps it
    assert np.isclose(np.sum(N.up2(y) * x), np.sum(y * N.up2_backward(x)), rtol=1e-12)
    assert np.allclose(N.avgpool2(x), N.up2_backward(x) / 8.0)
    assert np.allclose(N.avgpool2(np.full((4, 4, 4, 2), 3.5)), 3.5)
    assert np.isclose(np.sum(N.avgpool2(x) * y), np.sum(x * N.avgpool2_backward(y)), rtol=1e-12)
    assert N.up2(y)[3, 5, 1, 2] == y[1, 2, 0, 2]


def test_network_gradient_matches_finite_differences():
    """The whole U-Net's parameter gradients (every level, the skip paths and the head) against
    central differences of the loss, on an 8^3 input (the smallest for four levels)."""
    g = rng(5)
    p = N.init_params(7)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * g.standard_normal(p[k].shape)
    x0 = g.standard_normal((8, 8, 8, N.IN_CH))
    e = g.standard_normal((8, 8, 8, N.OUT_CH))
    y, cache = N.forward(p, x0, keep=True)
    L0, dy = N.loss_mse(y, e)
    grads = N.backward(p, cache, dy)
    assert set(grads) == set(p)
    hstep = 1e-6
    checked = 0
    for name, idx in [("e1a.w", (3, 13, 0)), ("e1b.b", (5,)), ("e2a.w", (7, 4, 9)),
                      ("e3b.w", (1, 22, 40)), ("ba.w", (100, 13, 3)), ("bb.b", (17,)),
                      ("d3a.w", (2, 13, 150)), ("d3a.w", (2, 13, 10)), ("d2b.w", (9, 0, 31)),
                      ("d1a.w", (4, 26, 40)), ("d1a.w", (4, 26, 3)), ("head.w", (1, 7)),
                      ("head.b", (0,))]:
        q = {k: v.copy() for k, v in p.items()}
        q[name][idx] += hstep
        Lp, _ = N.loss_mse(N.forward(q, x0), e)
        q[name][idx] -= 2 * hstep
        Lm, _ = N.loss_mse(N.forward(q, x0), e)
        fd = (Lp - Lm) / (2 * hstep)
        assert np.isclose(fd, grads[name][idx], rtol=2e-5, atol=1e-9), (name, idx, fd,
                                                                           grads[name][idx])
        checked += 1
    assert checked == 13


def test_bf16_rounding_against_torch_and_ties():
    torch = pytest.importorskip("torch")
    g = rng(6)
    x = (g.standard_normal(4096) * np.exp(g.uniform(-20, 20, 4096))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(N.bf16_round(x), ref)
    # ties go to the even neighbour: 1 + 2^-8 -> 1, 1 + 3 * 2^-8 -> 1 + 2^-6
    t = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.0 - 2.0 ** -7], dtype=np.float32)
    assert np.array_equal(N.bf16_round(t), np.array([1.0, 1.0 + 2.0 ** -6, -2.0],
                                                    dtype=np.float32))


def test_adam_first_step_closed_form():
    """From zero moments, the bias-corrected first Adam step is lr * g / (|g| + eps)."""
    p = {"a": np.array([1.0, -2.0, 0.5])}
    gr = {"a": np.array([0.3, -4.0, 1e-3])}
    st = {}
    N.adam_step(p, gr, st, lr=0.01)
    ref = np.array([1.0, -2.0, 0.5]) - 0.01 * gr["a"] / (np.abs(gr["a"]) + 1e-8)
    assert np.allclose(p["a"], ref, rtol=1e-12)
    assert st["t"] == 1


def test_preconditioner_is_homogeneous():
    g = rng(8)
    p = N.init_params(3)
    r = g.standard_normal((8, 8, 8)) + 1j * g.standard_normal((8, 8, 8))
    med = g.uniform(0.3, 1.0, (8, 8, 8))
    z1 = N.apply_preconditioner(p, r, med)
    z2 = N.apply_preconditioner(p, 3.0 * r, med)
    assert np.allclose(z2, 3.0 * z1, rtol=1e-12)
