"""The oracle's time discretisations (oracle.model.drug_step,
oracle.model.o2_transient_step; implicit Euler and Crank-Nicolson, Section
2.4.1) pinned by closed forms: the amplification factor of a single discrete
Fourier mode, the order of accuracy against the exact solution of the linear
ODE system (matrix exponential), steady states, and the limits h -> infinity."""

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import model as M
from oracle import params as Pm
from oracle import stencil as S


def _dense_laplacian(shape):
    n = int(np.prod(shape))
    L = np.zeros((n, n))
    idx = np.arange(n).reshape(shape)
    for ax in range(len(shape)):
        a = np.moveaxis(idx, ax, 0)
        for i, j in zip(a[:-1].reshape(-1), a[1:].reshape(-1)):
            L[i, i] += 1; L[j, j] += 1; L[i, j] -= 1; L[j, i] -= 1
    return L


@pytest.mark.parametrize("scheme,m", [(0, 1), (1, 1), (1, 3), (0, 4)])
def test_fourier_mode_amplification(scheme, m):
    """No vessels, no uptake: a Neumann cosine mode of eigenvalue mu of A_0 is
    multiplied per sub-step by 1/(1 + h mu) (implicit Euler) or
    (2/h - mu)/(2/h + mu) (Crank-Nicolson)."""
    nz, ny, nx = 3, 4, 11
    cfg = Pm.Config(nx, ny, nz, n_drugs=1, drug_scheme=scheme, drug_substeps=m, rtol_drug=1e-14,
                    D_G=(50.0,) * 3, psi_G=(0.02,) * 3)
    st = np.zeros((nz, ny, nx), dtype=np.uint8)
    kx, ky = 3, 1
    x, y = np.arange(nx), np.arange(ny)
    mode = np.cos(np.pi * kx * (x + 0.5) / nx)[None, None, :] * np.cos(np.pi * ky * (y + 0.5) / ny)[None, :, None]
    mode = np.broadcast_to(mode, st.shape).copy()
    lam = (2 - 2 * np.cos(np.pi * kx / nx)) + (2 - 2 * np.cos(np.pi * ky / ny))
    mu = S.drug_coupling(cfg, 0) * lam + cfg.psi_G[0]
    h = cfg.dt / m
    g = 1 / (1 + h * mu) if scheme == 0 else (2 / h - mu) / (2 / h + mu)
    G, _ = M.drug_step(st, np.ones(st.shape), mode, 5, cfg, 0)
    assert np.max(np.abs(G - g ** m * mode)) <= 1e-12 * max(abs(g ** m), 1e-3)


def _exact_drug(st, perf, G0, cfg, T):
    """u(T) of du/dt = -A_0 u + kappa G_0(t) with G_0(t) = peak exp(-k t)
    (one bolus at t = 0): e^{-A_0 T} u0 + (A_0 - k)^{-1}(e^{-kT} - e^{-A_0 T}) kappa peak."""
    n = st.size
    A0 = S.drug_coupling(cfg, 0) * _dense_laplacian(st.shape) + np.diag(S.drug_reaction0(st, perf, cfg, 0).reshape(-1))
    E = expm(-A0 * T)
    k = cfg.plasma_decay[0]
    f = S.drug_kappa(st, perf, cfg, 0).reshape(-1) * cfg.dose_peak[0]
    part = np.linalg.solve(A0 - k * np.eye(n), (np.exp(-k * T) * np.eye(n) - E) @ f)
    return (E @ G0.reshape(-1) + part).reshape(st.shape)


@pytest.mark.parametrize("scheme,order", [(0, 1), (1, 2)])
def test_order_of_accuracy(scheme, order):
    shape = (3, 4, 4)
    rng = np.random.default_rng(5)
    st = np.where(rng.random(shape) < 0.2, Pm.VESSEL, Pm.PROLIF).astype(np.uint8)
    perf = rng.uniform(0.5, 1.5, shape)
    G0 = rng.uniform(0.0, 1.0, shape)
    base = dict(n_drugs=1, rtol_drug=1e-15, D_G=(10.0,) * 3, psi_G=(0.01,) * 3, kappa_G=(0.05,) * 3,
                uptake_G=(0.003,) * 3, plasma_decay=(0.01,) * 3, dose_interval=1000)
    ref = _exact_drug(st, perf, G0, Pm.Config(4, 4, 3, **base), 60.0)
    errs = []
    for m in (32, 64, 128):
        cfg = Pm.Config(4, 4, 3, drug_scheme=scheme, drug_substeps=m, **base)
        G, _ = M.drug_step(st, perf, G0, 0, cfg, 0)
        errs.append(np.max(np.abs(G - ref)))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    for r in ratios:
        assert 2 ** order * 0.85 <= r <= 2 ** order * 1.15, (errs, ratios)


def test_steady_states_are_kept():
    shape = (4, 5, 6)
    rng = np.random.default_rng(6)
    st = rng.integers(0, 6, size=shape).astype(np.uint8)
    st.reshape(-1)[0] = Pm.VESSEL
    perf = rng.uniform(0.5, 1.5, shape)
    # drug with constant plasma (no decay, one bolus): u* = A_0^{-1} kappa peak
    for scheme in (0, 1):
        cfg = Pm.Config(6, 5, 4, n_drugs=1, drug_scheme=scheme, drug_substeps=3, rtol_drug=1e-14,
                        plasma_decay=(0.0,) * 3, dose_interval=10 ** 6)
        A0 = S.drug_coupling(cfg, 0) * _dense_laplacian(shape) + np.diag(S.drug_reaction0(st, perf, cfg, 0).reshape(-1))
        ustar = np.linalg.solve(A0, S.drug_kappa(st, perf, cfg, 0).reshape(-1) * cfg.dose_peak[0]).reshape(shape)
        G, _ = M.drug_step(st, perf, ustar, 2, cfg, 0)
        assert np.max(np.abs(G - ustar)) <= 1e-11 * np.max(np.abs(ustar))
    # oxygen: the nonlinear quasi-steady field is a fixed point of both time schemes
    Kq, _ = M.o2_picard(st, np.full(shape, 20.0), Pm.Config(6, 5, 4, picard_tol=1e-14, rtol_o2=1e-14))
    for scheme in (1, 2):
        cfg = Pm.Config(6, 5, 4, o2_scheme=scheme, o2_substeps=2, rtol_o2=1e-14)
        K, _ = M.o2_transient_step(st, Kq, cfg)
        assert np.max(np.abs(K - Kq)) <= 1e-10 * np.max(Kq)


def test_large_step_limits():
    """h -> infinity: implicit Euler reduces to the quasi-steady linearised
    solve; Crank-Nicolson to K + K_old = 2 A^{-1} f (A linearised about K_old)."""
    shape = (4, 5, 6)
    rng = np.random.default_rng(7)
    st = rng.integers(0, 6, size=shape).astype(np.uint8)
    st.reshape(-1)[0] = Pm.VESSEL
    K_old = rng.uniform(0.0, 20.0, shape)
    qs, _ = M.o2_solve(st, K_old, Pm.Config(6, 5, 4, rtol_o2=1e-14))
    cfg = Pm.Config(6, 5, 4, dt=1e15, rtol_o2=1e-14)
    K_ie, _ = M.o2_transient_step(st, K_old, Pm.Config(**{**cfg.__dict__, "o2_scheme": 1}))
    K_cn, _ = M.o2_transient_step(st, K_old, Pm.Config(**{**cfg.__dict__, "o2_scheme": 2}))
    assert np.max(np.abs(K_ie - qs)) <= 1e-9 * np.max(qs)
    assert np.max(np.abs(K_cn + K_old - 2 * qs)) <= 1e-9 * np.max(qs)


def test_transient_oxygen_relaxes_to_quasi_steady():
    """Many short implicit-Euler steps from K = K0 relax to the nonlinear
    quasi-steady field (the Picard fixed point)."""
    shape = (4, 5, 6)
    rng = np.random.default_rng(8)
    st = rng.integers(0, 6, size=shape).astype(np.uint8)
    st.reshape(-1)[0] = Pm.VESSEL
    Kq, _ = M.o2_picard(st, np.full(shape, 20.0), Pm.Config(6, 5, 4, picard_tol=1e-13, rtol_o2=1e-14))
    cfg = Pm.Config(6, 5, 4, o2_scheme=1, o2_substeps=200, dt=2.0, rtol_o2=1e-13)
    K = np.full(shape, 20.0)
    K, _ = M.o2_transient_step(st, K, cfg)
    assert np.max(np.abs(K - Kq)) <= 1e-8 * np.max(Kq)
