"""CPU oracle of the learned right preconditioner (test infrastructure, like all of oracle/).

The paper has no network; this is the variable right preconditioner that flexible GMRES admits
(Section 2, the remark after Algorithm 1: FGMRES allows the preconditioner to change from step
to step).  Everything here is a plain definition in float64 numpy, for checking the library's
BF16 tensor-core kernels; nothing in it is tuned.  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may use it.

Layout: a feature map is a float array x[D, H, W, C] (channels last, z slowest); a 3x3x3
convolution weight is w[co, t, ci] with tap t = 9 dz + 3 dy + dx, dz, dy, dx in {0, 1, 2}
standing for the offsets -1, 0, +1 along z, y, x; zero padding of one voxel ("same" size).

Network (a 4-level U-Net, 16 base channels, 3x3x3 kernels):
  input  x0: [D, H, W, 8]  (channel 0: Re r, 1: Im r, 2: the medium channel, 3..7: zero)
  enc1:  conv 8->16, relu, conv 16->16, relu                 -> s1   (D)
  enc2:  avgpool2, conv 16->32, relu, conv 32->32, relu       -> s2   (D/2)
  enc3:  avgpool2, conv 32->64, relu, conv 64->64, relu       -> s3   (D/4)
  bott:  avgpool2, conv 64->128, relu, conv 128->128, relu    -> b    (D/8)
  dec3:  up2(b) ++ s3 (192), conv ->64, relu, conv 64->64, relu
  dec2:  up2 ++ s2 (96), conv ->32, relu, conv 32->32, relu
  dec1:  up2 ++ s1 (48), conv ->16, relu, conv 16->16, relu
  head:  1x1x1 conv 16 -> 2 (no activation): (Re e, Im e)
where "++" is concatenation along channels (upsampled map first), avgpool2 the mean over 2x2x2
blocks and up2 nearest-neighbour repetition.  Every 3x3x3 convolution has a bias.
"""
from __future__ import annotations

import numpy as np

LEVELS = (16, 32, 64, 128)
IN_CH = 8
OUT_CH = 2


# ------------------------------------------------------------------------- number formats
def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float32.
    bfloat16 keeps the top 16 bits of the float32 encoding; NaN and Inf are not expected."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


# ------------------------------------------------------------------------- layers
def tap_offsets():
    """(dz, dy, dx) offsets of the 27 taps in tap order t = 9 dz + 3 dy + dx."""
    return [(dz - 1, dy - 1, dx - 1) for dz in range(3) for dy in range(3) for dx in range(3)]


def shifted(x: np.ndarray, oz: int, oy: int, ox: int) -> np.ndarray:
    """y[z, y, x] = x[z + oz, y + oy, x + ox], zero outside the map."""
    D, H, W = x.shape[:3]
    y = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -oz), min(D, D - oz)), slice(max(0, -oy), min(H, H - oy)), \
        slice(max(0, -ox), min(W, W - ox))
    zt, yt, xt = slice(max(0, oz), min(D, D + oz)), slice(max(0, oy), min(H, H + oy)), \
        slice(max(0, ox), min(W, W + ox))
    y[zs, ys, xs] = x[zt, yt, xt]
    return y


def conv3(x: np.ndarray, w: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """3x3x3 'same' convolution (cross-correlation) in float64:
    out[v, co] = sum_t sum_ci x[v + off_t, ci] w[co, t, ci] + b[co]."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (oz, oy, ox) in enumerate(tap_offsets()):
        out += shifted(x, oz, oy, ox) @ w[:, t, :].T
    if b is not None:
        out += np.asarray(b, dtype=np.float64)
    return out


def conv3_backward(x: np.ndarray, w: np.ndarray, dout: np.ndarray):
    """Gradients of conv3 with respect to its input, weight and bias, given d(loss)/d(out)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dout = np.asarray(dout, dtype=np.float64)
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    Cin = x.shape[3]
    for t, (oz, oy, ox) in enumerate(tap_offsets()):
        xs = shifted(x, oz, oy, ox)
        dw[:, t, :] = dout.reshape(-1, dout.shape[3]).T @ xs.reshape(-1, Cin)
        # out depends on x[v + off] through w: dx[u] += dout[u - off] w
        dx += shifted(dout @ w[:, t, :], -oz, -oy, -ox)
    db = dout.reshape(-1, dout.shape[3]).sum(axis=0)
    return dx, dw, db


def conv1(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """1x1x1 convolution: out[v, co] = sum_ci x[v, ci] w[co, ci] + b[co]."""
    return np.asarray(x, dtype=np.float64) @ np.asarray(w, dtype=np.float64).T + b


def conv1_backward(x, w, dout):
    x = np.asarray(x, dtype=np.float64)
    dout = np.asarray(dout, dtype=np.float64)
    dx = dout @ np.asarray(w, dtype=np.float64)
    dw = dout.reshape(-1, dout.shape[3]).T @ x.reshape(-1, x.shape[3])
    db = dout.reshape(-1, dout.shape[3]).sum(axis=0)
    return dx, dw, db


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x: np.ndarray) -> np.ndarray:
    """Mean over 2x2x2 blocks (even sizes)."""
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def avgpool2_backward(dout: np.ndarray) -> np.ndarray:
    return up2(dout) / 8.0


def up2(x: np.ndarray) -> np.ndarray:
    """Nearest-neighbour upsampling by 2 along z, y and x."""
    return np.repeat(np.repeat(np.repeat(x, 2, axis=0), 2, axis=1), 2, axis=2)


def up2_backward(dout: np.ndarray) -> np.ndarray:
    D, H, W, C = dout.shape
    return dout.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


# ------------------------------------------------------------------------- the network
def conv_names():
    """The 3x3x3 convolutions of the network in order, with (C_in, C_out)."""
    c1, c2, c3, c4 = LEVELS
    return [("e1a", IN_CH, c1), ("e1b", c1, c1), ("e2a", c1, c2), ("e2b", c2, c2),
            ("e3a", c2, c3), ("e3b", c3, c3), ("ba", c3, c4), ("bb", c4, c4),
            ("d3a", c4 + c3, c3), ("d3b", c3, c3), ("d2a", c3 + c2, c2), ("d2b", c2, c2),
            ("d1a", c2 + c1, c1), ("d1b", c1, c1)]


def init_params(seed: int) -> dict:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases; head weights std 1/sqrt(16)."""
    g = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, ci, co in conv_names():
        p[name + ".w"] = g.standard_normal((co, 27, ci)) * np.sqrt(2.0 / (27 * ci))
        p[name + ".b"] = np.zeros(co)
    p["head.w"] = g.standard_normal((OUT_CH, LEVELS[0])) / np.sqrt(LEVELS[0])
    p["head.b"] = np.zeros(OUT_CH)
    return p


def _identity(x):
    return x


def forward(p: dict, x0: np.ndarray, keep: bool = False, bf16: bool = False):
    """Network output y[D, H, W, 2] for the input map x0[D, H, W, 8] (D, H, W multiples of 8).
    keep: also return every intermediate map, for the backward pass.  bf16: round the input,
    the 3x3x3 weights and every stored feature map (ReLU and pooling outputs) to bfloat16, the
    storage format of a reduced-precision implementation; the arithmetic stays float64."""
    q = bf16_round if bf16 else _identity
    x0 = q(x0)
    cache = {"x0": x0, "bf16": bf16}

    def cr(name, x):  # conv + relu, keeping the input and the output
        cache[name + ".in"] = x
        y = q(relu(conv3(x, q(p[name + ".w"]), p[name + ".b"])))
        cache[name + ".out"] = y
        return y

    s1 = cr("e1b", cr("e1a", x0))
    s2 = cr("e2b", cr("e2a", q(avgpool2(s1))))
    s3 = cr("e3b", cr("e3a", q(avgpool2(s2))))
    b = cr("bb", cr("ba", q(avgpool2(s3))))
    d3 = cr("d3b", cr("d3a", np.concatenate([up2(b), s3], axis=3)))
    d2 = cr("d2b", cr("d2a", np.concatenate([up2(d3), s2], axis=3)))
    d1 = cr("d1b", cr("d1a", np.concatenate([up2(d2), s1], axis=3)))
    cache["head.in"] = d1
    y = conv1(d1, p["head.w"], p["head.b"])
    return (y, cache) if keep else y


def backward(p: dict, cache: dict, dy: np.ndarray) -> dict:
    """Gradients of a loss with respect to every parameter, given d(loss)/dy.  After a bf16
    forward pass, the gradient through each ReLU and the weights of each data gradient are
    rounded to bfloat16 as well (the operands of a reduced-precision backward pass); the bias
    gradient is the sum of the unrounded values."""
    q = bf16_round if cache.get("bf16") else _identity
    grads = {}
    dd1, grads["head.w"], grads["head.b"] = conv1_backward(cache["head.in"], p["head.w"], dy)

    def cr_back(name, dout):  # through relu, then the convolution
        dpre = dout * (cache[name + ".out"] > 0)
        db = dpre.reshape(-1, dpre.shape[3]).sum(axis=0)
        dx, grads[name + ".w"], _ = conv3_backward(cache[name + ".in"], q(p[name + ".w"]),
                                                   q(dpre))
        grads[name + ".b"] = db
        return dx

    c1, c2, c3, c4 = LEVELS
    dcat1 = cr_back("d1a", cr_back("d1b", dd1))
    dd2, ds1 = up2_backward(dcat1[..., :c2]), dcat1[..., c2:]
    dcat2 = cr_back("d2a", cr_back("d2b", dd2))
    dd3, ds2 = up2_backward(dcat2[..., :c3]), dcat2[..., c3:]
    dcat3 = cr_back("d3a", cr_back("d3b", dd3))
    db, ds3 = up2_backward(dcat3[..., :c4]), dcat3[..., c4:]
    ds3 = ds3 + avgpool2_backward(cr_back("ba", cr_back("bb", db)))
    ds2 = ds2 + avgpool2_backward(cr_back("e3a", cr_back("e3b", ds3)))
    ds1 = ds1 + avgpool2_backward(cr_back("e2a", cr_back("e2b", ds2)))
    cr_back("e1a", cr_back("e1b", ds1))
    return grads


def loss_mse(y: np.ndarray, e: np.ndarray):
    """L = sum (y - e)^2 / (2 N) over the N voxels; returns (L, dL/dy)."""
    nvox = y.shape[0] * y.shape[1] * y.shape[2]
    d = y - e
    return float(np.sum(d * d) / (2.0 * nvox)), d / nvox


def adam_step(p: dict, grads: dict, state: dict, lr: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update (Kingma and Ba, 2015) with bias correction, in place.  state holds the
    step count "t" and the moments "m.<name>", "v.<name>"."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k, gk in grads.items():
        m = state.get("m." + k, np.zeros_like(gk))
        v = state.get("v." + k, np.zeros_like(gk))
        m = beta1 * m + (1.0 - beta1) * gk
        v = beta2 * v + (1.0 - beta2) * gk * gk
        state["m." + k], state["v." + k] = m, v
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


# ------------------------------------------------------------------------- preconditioner use
def net_input(r: np.ndarray, medium: np.ndarray) -> np.ndarray:
    """The network's input map for a complex residual r[D, H, W] (scaled to unit RMS) and the
    medium channel: [Re r, Im r, medium, 0, 0, 0, 0, 0]."""
    x = np.zeros(r.shape + (IN_CH,))
    x[..., 0] = r.real
    x[..., 1] = r.imag
    x[..., 2] = medium
    return x


def apply_preconditioner(p: dict, r: np.ndarray, medium: np.ndarray) -> np.ndarray:
    """z = N(r): the network applied to r scaled to unit RMS, the output scaled back (the map
    r -> z is then homogeneous of degree 1, as a preconditioner must be for FGMRES)."""
    rms = float(np.sqrt(np.mean(np.abs(r) ** 2)))
    if rms == 0.0:
        return np.zeros_like(r)
    y = forward(p, net_input(r / rms, medium))
    return rms * (y[..., 0] + 1j * y[..., 1])
