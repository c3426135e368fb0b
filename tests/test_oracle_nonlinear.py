"""The nonlinear quasi-steady oxygen solve of the oracle (oracle.model.o2_picard)
pinned against the nonlinear equation itself and against a dense Newton
iteration written here."""

import numpy as np

from oracle import model as M
from oracle import params as Pm
from oracle import stencil as S


def _lattice(shape, seed):
    rng = np.random.default_rng(seed)
    st = rng.integers(0, 6, size=shape).astype(np.uint8)
    st.reshape(-1)[0] = Pm.VESSEL
    return st


def test_picard_fixed_point_solves_the_nonlinear_equation():
    cfg = Pm.Config(6, 5, 4, picard_tol=1e-12, rtol_o2=1e-13)
    st = _lattice((4, 5, 6), 1)
    K, it = M.o2_picard(st, np.full(st.shape, cfg.K0), cfg)
    F = M.o2_residual_nonlinear(st, K, cfg)
    scale = cfg.r_K * cfg.K0
    assert it < cfg.picard_maxit
    assert np.max(np.abs(F)) <= 1e-8 * scale


def test_picard_matches_dense_newton():
    cfg = Pm.Config(5, 4, 3, picard_tol=1e-13, rtol_o2=1e-14)
    st = _lattice((3, 4, 5), 2)
    n = st.size
    cpl = S.o2_coupling(cfg)
    L = np.zeros((n, n))
    idx = np.arange(n).reshape(st.shape)
    for ax in range(3):
        a = np.moveaxis(idx, ax, 0)
        for i, j in zip(a[:-1].reshape(-1), a[1:].reshape(-1)):
            L[i, i] += 1; L[j, j] += 1; L[i, j] -= 1; L[j, i] -= 1
    cons = np.isin(st, (Pm.PROLIF, Pm.QUIESC, Pm.STROMA)).reshape(-1)
    ves = (st == Pm.VESSEL).reshape(-1)
    K = np.full(n, cfg.K0)
    for _ in range(50):     # Newton on F(K) = cpl L K + phi K/(K1+K)[c] + r_K (K - K0)[v]
        F = cpl * L @ K + np.where(cons, cfg.phi_K * K / (cfg.K1 + K), 0) + np.where(ves, cfg.r_K * (K - cfg.K0), 0)
        J = cpl * L + np.diag(np.where(cons, cfg.phi_K * cfg.K1 / (cfg.K1 + K) ** 2, 0) + np.where(ves, cfg.r_K, 0))
        dK = np.linalg.solve(J, -F)
        K += dK
        if np.max(np.abs(dK)) < 1e-14 * np.max(np.abs(K)):
            break
    Kp, _ = M.o2_picard(st, np.full(st.shape, cfg.K0), cfg)
    assert np.max(np.abs(Kp.reshape(-1) - K)) <= 1e-10 * np.max(np.abs(K))


def test_linearised_solve_keeps_the_nonlinear_solution_fixed():
    cfg = Pm.Config(6, 5, 4, picard_tol=1e-13, rtol_o2=1e-14)
    st = _lattice((4, 5, 6), 3)
    Knl, _ = M.o2_picard(st, np.full(st.shape, cfg.K0), cfg)
    Klin, _ = M.o2_solve(st, Knl, cfg)
    assert np.max(np.abs(Klin - Knl)) <= 1e-10 * np.max(np.abs(Knl))
