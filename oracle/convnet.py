"""FP64 reference of the learned oxygen warm-start network (no paper counterpart).

Test infrastructure only: nothing on the product path imports this module.

The paper warm-starts nothing; the GPU path can replace the previous-step
oxygen field as the CG initial guess of Eq. (oxygen) by
K_prev + (K0 / NET_SCALE) f(x), where f is a small 3-D convolutional
encoder-decoder and x holds, per site, the one-hot state code (6 channels),
the perfusion map, K_prev / K0 and the Jacobi-scaled initial residual
NET_SCALE (b - A K_prev) / (diag(A) K0) of the linearised operator (9
channels, zero-padded to 16).  This module is the plain FP64 definition of f,
of its gradients and of Adam, used to check the GPU kernels.  Activations are
stored in BF16 on the GPU; ``forward(..., bf16=True)`` rounds them at the
same points (the definition of the BF16 network), FP64 everywhere else.

Layout: activations (D, H, W, C) (channels last); a 3x3x3 weight tensor is
(27, C_out, C_in) with tap t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1); padding is
"same" with zeros.

Architecture (levels 0..3 with C = 16, 32, 64, 64; every spatial size must
be divisible by 8):
  e0 = relu(conv(x) + b)                  16
  e1 = relu(conv(pool(e0)) + b)           32
  e2 = relu(conv(pool(e1)) + b)           64
  e3 = relu(conv(pool(e2)) + b)           64
  d2 = relu(conv(up(e3)) + b + e2)        64
  d1 = relu(conv(up(d2)) + b + e1)        32
  d0 = relu(conv(up(d1)) + b + e0)        16
  out = d0 . w_head + b_head              1
pool = 2x2x2 average, up = 2x nearest.  Loss = mean((out - target)^2).
"""

from __future__ import annotations

import numpy as np

from . import stencil as S

IN_CH = 16
NET_SCALE = 64.0
LEVEL_CH = (16, 32, 64, 64)
# (name, C_in, C_out) of the seven 3x3x3 convolutions, in order
CONVS = (("enc0", IN_CH, 16), ("enc1", 16, 32), ("enc2", 32, 64), ("enc3", 64, 64),
         ("dec2", 64, 64), ("dec1", 64, 32), ("dec0", 32, 16))
OFFSETS = tuple((dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1))


def shift(x, dz, dy, dx):
    """y[z, y, x] = x[z + dz, y + dy, x + dx] with zeros outside (channels last)."""
    out = np.zeros_like(x)
    D, H, W = x.shape[:3]
    zs, ys, xs = slice(max(0, -dz), D - max(0, dz)), slice(max(0, -dy), H - max(0, dy)), slice(max(0, -dx), W - max(0, dx))
    zt, yt, xt = slice(max(0, dz), D - max(0, -dz)), slice(max(0, dy), H - max(0, -dy)), slice(max(0, dx), W - max(0, -dx))
    out[zs, ys, xs] = x[zt, yt, xt]
    return out


def conv3(x, w):
    """'same' 3x3x3 convolution: y[m, co] = sum_t sum_ci x[m + off_t, ci] w[t, co, ci]."""
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        y += shift(x, dz, dy, dx) @ w[t].T
    return y


def conv3_dgrad(gy, w):
    """Gradient of conv3 with respect to its input."""
    gx = np.zeros(gy.shape[:3] + (w.shape[2],))
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        gx += shift(gy, -dz, -dy, -dx) @ w[t]
    return gx


def conv3_wgrad(x, gy):
    """Gradient of conv3 with respect to its weights, shape (27, C_out, C_in)."""
    C = x.shape[-1]
    gw = np.zeros((27, gy.shape[-1], C))
    g2 = gy.reshape(-1, gy.shape[-1])
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        gw[t] = g2.T @ shift(x, dz, dy, dx).reshape(-1, C)
    return gw


def pool(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def pool_grad(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_grad(g):
    D, H, W, C = g.shape
    return g.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(rng):
    """He-normal weights, zero biases (FP64)."""
    p = {}
    for name, ci, co in CONVS:
        p[name + ".w"] = rng.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27 * ci))
        p[name + ".b"] = np.zeros(co)
    p["head.w"] = rng.standard_normal(16) * np.sqrt(1.0 / 16)
    p["head.b"] = np.zeros(1)
    return p


def forward(p, x, bf16=False):
    """Returns (out (D, H, W), cache of activations).

    With bf16=True the input, every stored activation and the convolution
    weights are rounded to BF16 (sums stay FP64); pooled tensors are rounded
    after the average.
    """
    r = bf16_round if bf16 else (lambda v: v)
    if bf16:
        p = {k: (bf16_round(v) if k.endswith(".w") and k != "head.w" else v) for k, v in p.items()}
    c = {"x": r(x)}
    relu = lambda v: r(np.maximum(v, 0.0))
    pool_r = lambda v: r(pool(v))
    c["e0"] = relu(conv3(c["x"], p["enc0.w"]) + p["enc0.b"])
    c["p0"] = pool_r(c["e0"])
    c["e1"] = relu(conv3(c["p0"], p["enc1.w"]) + p["enc1.b"])
    c["p1"] = pool_r(c["e1"])
    c["e2"] = relu(conv3(c["p1"], p["enc2.w"]) + p["enc2.b"])
    c["p2"] = pool_r(c["e2"])
    c["e3"] = relu(conv3(c["p2"], p["enc3.w"]) + p["enc3.b"])
    c["u3"] = up(c["e3"])
    c["d2"] = relu(conv3(c["u3"], p["dec2.w"]) + p["dec2.b"] + c["e2"])
    c["u2"] = up(c["d2"])
    c["d1"] = relu(conv3(c["u2"], p["dec1.w"]) + p["dec1.b"] + c["e1"])
    c["u1"] = up(c["d1"])
    c["d0"] = relu(conv3(c["u1"], p["dec0.w"]) + p["dec0.b"] + c["e0"])
    out = c["d0"] @ p["head.w"] + p["head.b"][0]
    c["params"] = p
    return out, c


def loss(out, target):
    return float(np.mean((out - target) ** 2))


def backward(p, c, gout, bf16=False, record=None):
    """Gradients of sum(out * gout) with respect to every parameter.

    Uses the (possibly BF16-rounded) weights the forward pass used.  With
    bf16=True the gradient with respect to each convolution's output (after
    the ReLU mask and, on the encoder side, after adding the skip path's
    gradient) is rounded to BF16 where it is formed: the BF16 network stores
    these tensors in BF16, as it stores its activations.  record (a dict), if
    given, receives each convolution's output gradient (as used) and input
    under the convolution's name, for checks of the weight gradients.
    """
    p = c.get("params", p)
    r = bf16_round if bf16 else (lambda v: v)
    g = {}

    def wgrad(name, x, gy):
        if record is not None:
            record[name] = (x, gy)
        g[name + ".w"] = conv3_wgrad(x, gy)
        g[name + ".b"] = gy.sum(axis=(0, 1, 2))

    g["head.w"] = c["d0"].reshape(-1, 16).T @ gout.reshape(-1)
    g["head.b"] = np.array([gout.sum()])
    gd0 = r((gout[..., None] * p["head.w"]) * (c["d0"] > 0))
    wgrad("dec0", c["u1"], gd0)
    ge0 = gd0.copy()
    gd1 = r(up_grad(conv3_dgrad(gd0, p["dec0.w"])) * (c["d1"] > 0))
    wgrad("dec1", c["u2"], gd1)
    ge1 = gd1.copy()
    gd2 = r(up_grad(conv3_dgrad(gd1, p["dec1.w"])) * (c["d2"] > 0))
    wgrad("dec2", c["u3"], gd2)
    ge2 = gd2.copy()
    ge3 = r(up_grad(conv3_dgrad(gd2, p["dec2.w"])) * (c["e3"] > 0))
    wgrad("enc3", c["p2"], ge3)
    ge2 = r((ge2 + pool_grad(conv3_dgrad(ge3, p["enc3.w"]))) * (c["e2"] > 0))
    wgrad("enc2", c["p1"], ge2)
    ge1 = r((ge1 + pool_grad(conv3_dgrad(ge2, p["enc2.w"]))) * (c["e1"] > 0))
    wgrad("enc1", c["p0"], ge1)
    ge0 = r((ge0 + pool_grad(conv3_dgrad(ge1, p["enc1.w"]))) * (c["e0"] > 0))
    wgrad("enc0", c["x"], ge0)
    return g


def mse_grad(out, target):
    """Loss mean((out - target)^2) and its gradient with respect to out."""
    n = out.size
    return float(np.mean((out - target) ** 2)), 2.0 * (out - target) / n


def residual_loss(out, target, state, K_prev, cfg):
    """Loss mean((A e)^2) / c^2 and its gradient with respect to out, where
    e = out - target, A is the oxygen operator of Eq. (oxygen) linearised
    about K_prev (the operator of the solve the guess starts) and
    c = D_K / dx^2.  Since A K_new = b, A e is the residual of the guess up
    to the output scale: the loss trains the quantity the solver's fallback
    test compares."""
    cpl = S.o2_coupling(cfg)
    reac = S.o2_reaction(state, K_prev, cfg)
    e = np.asarray(out, dtype=np.float64) - target
    u = S.apply_operator(e, cpl, reac) / cpl
    n = e.size
    return float(np.mean(u * u)), 2.0 * S.apply_operator(u, cpl, reac) / (cpl * n)


def adam(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1; returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def make_input(state, perf, K_prev, cfg):
    """The 16-channel input of the network for one oxygen solve.

    state is the lattice the solve sees, K_prev the previous oxygen field,
    which both linearises the consumption term (Section 2.4.1) and is the
    plain warm start.  Channel 8 is the Jacobi-scaled residual of K_prev for
    the operator of Eq. (oxygen), scaled by NET_SCALE / K0.
    """
    state = np.asarray(state)
    K_prev = np.asarray(K_prev, dtype=np.float64)
    D, H, W = state.shape
    x = np.zeros((D, H, W, IN_CH))
    for s in range(6):
        x[..., s] = state == s
    x[..., 6] = perf
    x[..., 7] = K_prev / cfg.K0
    reac = S.o2_reaction(state, K_prev, cfg)
    cpl = S.o2_coupling(cfg)
    r0 = S.o2_rhs(state, cfg) - S.apply_operator(K_prev, cpl, reac)
    x[..., 8] = NET_SCALE * r0 / (S.jacobi_diagonal(state.shape, cpl, reac) * cfg.K0)
    return x


def guess(K_prev, out, cfg):
    """The warm start K_prev + (K0 / NET_SCALE) f(x)."""
    return np.asarray(K_prev, dtype=np.float64) + (cfg.K0 / NET_SCALE) * out


def target(K_prev, K_new, cfg):
    """The training target: NET_SCALE (K_new - K_prev) / K0."""
    return NET_SCALE * (np.asarray(K_new, dtype=np.float64) - K_prev) / cfg.K0
