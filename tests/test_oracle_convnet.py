"""Pins of the FP64 network oracle (oracle/convnet.py) against definitions
that do not share its code: brute-force loops, scipy's correlate, adjoint
identities and central finite differences of the loss."""

import numpy as np
import pytest
from scipy import ndimage

from oracle import convnet as C
from oracle import params as Pm
from oracle import stencil as S


def brute_conv(x, w):
    D, H, W, CI = x.shape
    CO = w.shape[1]
    y = np.zeros((D, H, W, CO))
    for z in range(D):
        for yy in range(H):
            for xx in range(W):
                for t, (dz, dy, dx) in enumerate(C.OFFSETS):
                    zz, y2, x2 = z + dz, yy + dy, xx + dx
                    if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                        for co in range(CO):
                            for ci in range(CI):
                                y[z, yy, xx, co] += x[zz, y2, x2, ci] * w[t, co, ci]
    return y


def test_conv_matches_brute_force_loops(rng):
    x = rng.standard_normal((3, 4, 5, 2))
    w = rng.standard_normal((27, 3, 2))
    assert np.allclose(C.conv3(x, w), brute_conv(x, w), rtol=0, atol=1e-12)


def test_conv_matches_scipy_correlate(rng):
    x = rng.standard_normal((5, 6, 7, 3))
    w = rng.standard_normal((27, 2, 3))
    y = C.conv3(x, w)
    for co in range(2):
        ref = np.zeros(x.shape[:3])
        for ci in range(3):
            k = w[:, co, ci].reshape(3, 3, 3)           # [dz+1, dy+1, dx+1]
            ref += ndimage.correlate(x[..., ci], k, mode="constant", cval=0.0)
        assert np.allclose(y[..., co], ref, atol=1e-12)


def test_single_tap_is_a_shift(rng):
    x = rng.standard_normal((4, 4, 4, 1))
    w = np.zeros((27, 1, 1))
    t = C.OFFSETS.index((1, 0, -1))
    w[t, 0, 0] = 1.0
    y = C.conv3(x, w)[..., 0]
    # y[z, y, x] = x[z + 1, y, x - 1]
    assert y[1, 2, 3] == x[2, 2, 2, 0] and y[3, 0, 0] == 0.0 and y[0, 1, 2] == x[1, 1, 1, 0]


def test_adjoint_identities(rng):
    x = rng.standard_normal((4, 6, 8, 3))
    yc = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(C.pool(x) * yc), np.sum(x * C.pool_grad(yc)))
    assert np.isclose(np.sum(C.up(yc) * x), np.sum(yc * C.up_grad(x)))
    w = rng.standard_normal((27, 5, 3))
    gy = rng.standard_normal((4, 6, 8, 5))
    # <conv(x), gy> = <x, dgrad(gy)> = <w, wgrad(x, gy)>
    a = np.sum(C.conv3(x, w) * gy)
    assert np.isclose(a, np.sum(x * C.conv3_dgrad(gy, w)))
    assert np.isclose(a, np.sum(w * C.conv3_wgrad(x, gy)))
    assert np.allclose(C.pool(C.up(yc)), yc, rtol=1e-15, atol=0)


def test_bf16_rounding_special_values():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 0.0])
    assert np.array_equal(C.bf16_round(v), [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -2.5, 0.0])


def _loss_of(p, x, tgt, bf16=False):
    out, _ = C.forward(p, x, bf16=bf16)
    return C.loss(out, tgt)


def test_network_gradient_matches_finite_differences(rng):
    x = rng.standard_normal((8, 8, 8, C.IN_CH)) * 0.5
    p = C.init_params(rng)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    tgt = rng.standard_normal((8, 8, 8))
    out, cache = C.forward(p, x)
    _, gout = C.mse_grad(out, tgt)
    g = C.backward(p, cache, gout)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = _loss_of(p, x, tgt)
            flat[idx] = old - h
            lm = _loss_of(p, x, tgt)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (k, idx, fd, an)


def test_mse_gradient_and_adam_first_step():
    out = np.array([1.0, 2.0, 4.0])
    tgt = np.array([0.0, 2.0, 1.0])
    L, g = C.mse_grad(out, tgt)
    assert L == pytest.approx((1 + 0 + 9) / 3) and np.allclose(g, [2 / 3, 0, 2])
    # first Adam step moves each weight by lr * sign(g) (up to eps)
    w, m, v = C.adam(np.zeros(3), np.array([0.5, -2.0, 1e-3]), np.zeros(3), np.zeros(3), 1, 0.1)
    assert np.allclose(w, [-0.1, 0.1, -0.1], rtol=1e-4)


def test_input_features():
    cfg = Pm.Config(6, 5, 4)
    rng = np.random.default_rng(3)
    st = rng.integers(0, 6, size=(4, 5, 6)).astype(np.uint8)
    perf = rng.uniform(0.5, 1.5, size=st.shape)
    cpl = S.o2_coupling(cfg)
    K = rng.uniform(5, 20, size=st.shape)
    x = C.make_input(st, perf, K, cfg)
    assert np.array_equal(x[..., :6].argmax(-1), st) and np.all(x[..., 9:] == 0)
    assert np.array_equal(x[..., 6], perf) and np.allclose(x[..., 7], K / 20.0)
    assert np.any(np.abs(x[..., 8]) > 1e-3)

    # dense Picard iteration K <- A(K)^{-1} b to its fixed point: there the
    # residual channel, which lags the operator at K_prev itself, vanishes
    n = st.size
    b = np.where(st == Pm.VESSEL, cfg.r_K * cfg.K0, 0.0).reshape(-1)
    Kf = K.copy()
    for _ in range(60):
        cons = np.where(np.isin(st, (Pm.PROLIF, Pm.QUIESC, Pm.STROMA)), cfg.phi_K / (cfg.K1 + Kf), 0.0)
        reac = (cons + np.where(st == Pm.VESSEL, cfg.r_K, 0.0)).reshape(-1)
        A = np.diag(reac)
        idx = np.arange(n).reshape(st.shape)
        for ax in range(3):
            a = np.moveaxis(idx, ax, 0)
            for i, j in zip(a[:-1].reshape(-1), a[1:].reshape(-1)):
                A[i, i] += cpl; A[j, j] += cpl; A[i, j] -= cpl; A[j, i] -= cpl
        Kf = np.linalg.solve(A, b).reshape(st.shape)
    xf = C.make_input(st, perf, Kf, cfg)
    assert np.max(np.abs(xf[..., 8])) < 1e-9
    Kn = rng.uniform(5, 20, size=st.shape)
    assert np.allclose(C.guess(K, C.target(K, Kn, cfg), cfg), Kn)


def test_residual_loss_gradient_and_special_cases():
    cfg = Pm.Config(5, 4, 3)
    rng = np.random.default_rng(8)
    st = rng.integers(0, 6, size=(3, 4, 5)).astype(np.uint8)
    Kp = rng.uniform(5, 20, size=st.shape)
    out = rng.standard_normal(st.shape)
    tgt = rng.standard_normal(st.shape)
    L, g = C.residual_loss(out, tgt, st, Kp, cfg)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (2, 3, 4), (1, 0, 2)]:
        o = out.copy()
        o[idx] += h
        lp = C.residual_loss(o, tgt, st, Kp, cfg)[0]
        o[idx] -= 2 * h
        lm = C.residual_loss(o, tgt, st, Kp, cfg)[0]
        assert abs((lp - lm) / (2 * h) - g[idx]) <= 1e-6 * max(1.0, abs(g[idx]))
    # a constant error on a lattice without consumers or vessels lies in the
    # Neumann Laplacian's null space: zero loss
    st0 = np.zeros_like(st)
    assert C.residual_loss(tgt + 0.3, tgt, st0, Kp, cfg)[0] < 1e-24
    # a single-site error e at an isolated interior empty site: (A e)/c has
    # 6 e at the site and -e at each of its 6 neighbours -> mean = 42 e^2 / n
    st1 = np.zeros((3, 3, 3), dtype=np.uint8)
    e = np.zeros((3, 3, 3))
    e[1, 1, 1] = 0.5
    L1, _ = C.residual_loss(e, np.zeros_like(e), st1, np.ones_like(e), Pm.Config(3, 3, 3))
    assert L1 == pytest.approx(42 * 0.25 / 27)


def test_bf16_backward_rounds_the_activation_gradients_only():
    """backward(bf16=True): every recorded output gradient is a BF16 value,
    each weight gradient is the weight-gradient correlation of the recorded
    tensors, and the result stays within BF16 rounding of the exact backward."""
    rng = np.random.default_rng(3)
    p = C.init_params(rng)
    x = C.bf16_round(rng.standard_normal((8, 8, 8, C.IN_CH)))
    out, cache = C.forward(p, x, bf16=True)
    gout = rng.standard_normal(out.shape) / out.size
    rec = {}
    g16 = C.backward(p, cache, gout, bf16=True, record=rec)
    g64 = C.backward(p, cache, gout)
    for name, _, _ in C.CONVS:
        xin, gy = rec[name]
        assert np.array_equal(C.bf16_round(gy), gy), name
        assert np.allclose(g16[name + ".w"], C.conv3_wgrad(xin, gy), rtol=1e-13, atol=0)
        e = np.linalg.norm(g16[name + ".w"] - g64[name + ".w"]) / np.linalg.norm(g64[name + ".w"])
        assert 0 < e < 2 ** -6, (name, e)
    assert np.array_equal(g16["head.w"], g64["head.w"])
