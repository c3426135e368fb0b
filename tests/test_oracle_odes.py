"""Pins for the oracle's plasma levels and per-cell ODEs.

Checked against scipy's adaptive integrators (solve_ivp at rtol 1e-12), the
exact linear/exponential solutions, RK4's fourth-order convergence and its
error bound.
"""

import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import params as Pm
from oracle.odes import ode_update, p53_at, p53_rate, phi_advance, vegf_rk4
from oracle.plasma import plasma_concentration


@pytest.mark.parametrize("decay", [3.93e3 / 2430e3, 0.983e3 / 18e3])
def test_plasma_matches_integrated_boluses(decay):
    interval = 21 * 60.0
    peak = 1.0
    t_end = 3.5 * interval
    # integrate dG/dt = -k G between doses, adding the bolus at each dose time
    G = 0.0
    t = 0.0
    samples = {}
    checkpoints = [0.0, 60.0, 0.7 * interval, interval, interval + 1.0, 2 * interval + 600.0, t_end]
    dose_times = [n * interval for n in range(4)]
    for n, td in enumerate(dose_times):
        if td > t_end:
            break
        if td > t:
            sol = solve_ivp(lambda s, y: -decay * y, (t, td), [G], rtol=1e-12, atol=1e-15,
                            dense_output=True)
            for c in checkpoints:
                if t <= c < td:
                    samples[c] = sol.sol(c)[0]
            G = sol.y[0, -1]
            t = td
        G += peak
        if td in checkpoints:
            samples[td] = G
    sol = solve_ivp(lambda s, y: -decay * y, (t, t_end), [G], rtol=1e-12, atol=1e-15, dense_output=True)
    for c in checkpoints:
        if t <= c <= t_end and c not in samples:
            samples[c] = sol.sol(c)[0]
    for c, v in samples.items():
        assert math.isclose(plasma_concentration(c, peak, decay, interval), v, rel_tol=1e-9, abs_tol=1e-13), c


def test_plasma_before_first_dose_and_peak():
    assert plasma_concentration(-1.0, 1.0, 0.1, 100.0) == 0.0
    assert plasma_concentration(0.0, 2.5, 0.1, 100.0) == 2.5


CFG = Pm.Config(nx=1, ny=1, nz=1)


@pytest.mark.parametrize("K", [0.0, 0.5, 3.0, 20.0])
def test_phi_exact_linear(K):
    phi0 = 0.3
    sol = solve_ivp(lambda t, y: [K / (CFG.T_cycle * (CFG.K_phi + K))], (0, 60.0), [phi0],
                    rtol=1e-12, atol=1e-15)
    assert math.isclose(phi_advance(phi0, K, 60.0, CFG), sol.y[0, -1], rel_tol=1e-12)
    # exact at fixed K: two half steps equal one step
    half = phi_advance(phi_advance(phi0, K, 30.0, CFG), K, 30.0, CFG)
    assert math.isclose(half, phi_advance(phi0, K, 60.0, CFG), rel_tol=1e-15)


@pytest.mark.parametrize("K", [0.0, 0.004, 0.01, 2.0, 20.0])
@pytest.mark.parametrize("P0", [0.0, 0.05, 1.0])
def test_p53_exact_solution(K, P0):
    lam = p53_rate(np.array(K), CFG)
    sol = solve_ivp(lambda t, y: [CFG.k1 - CFG.k1p * K / (CFG.K_p53 + K) * y[0]], (0, 60.0), [P0],
                    rtol=1e-12, atol=1e-16, dense_output=True)
    for s in (0.0, 0.5, 17.0, 60.0):
        assert math.isclose(float(p53_at(P0, lam, s, CFG)), sol.sol(s)[0], rel_tol=1e-9, abs_tol=1e-14)


def coupled_reference(V0, P0, K, T):
    def f(t, y):
        P, V = y
        return [CFG.k1 - CFG.k1p * K / (CFG.K_p53 + K) * P,
                CFG.k2 + CFG.k2pp * P * V / (CFG.J5 + V) - CFG.k2p * K / (CFG.K_V + K) * V]
    return solve_ivp(f, (0, T), [P0, V0], method="DOP853", rtol=1e-13, atol=1e-16).y[1, -1]


@pytest.mark.parametrize("K", [0.0, 0.01, 1.0, 20.0])
@pytest.mark.parametrize("V0,P0", [(0.0, 0.0), (0.03, 0.2), (1.0, 5.0)])
def test_vegf_rk4_close_to_reference(K, V0, P0):
    ref = coupled_reference(V0, P0, K, 60.0)
    got = float(vegf_rk4(np.array(V0), np.array(P0), np.array(K), 60.0, 60, CFG))
    # RK4 with h = 1 min on rates <= 0.01/min: local error ~ (0.01 h)^5 / 120
    assert math.isclose(got, ref, rel_tol=1e-9, abs_tol=1e-14)


def test_vegf_rk4_fourth_order():
    # faster rates make the truncation error visible above rounding
    cfg = Pm.Config(nx=1, ny=1, nz=1, k2p=0.1, k2pp=-0.05, k1p=0.1)
    K, V0, P0, T = 2.0, 0.8, 1.5, 20.0

    def f(t, y):
        P, V = y
        return [cfg.k1 - cfg.k1p * K / (cfg.K_p53 + K) * P,
                cfg.k2 + cfg.k2pp * P * V / (cfg.J5 + V) - cfg.k2p * K / (cfg.K_V + K) * V]
    ref = solve_ivp(f, (0, T), [P0, V0], method="DOP853", rtol=1e-13, atol=1e-16).y[1, -1]
    errs = [abs(float(vegf_rk4(np.array(V0), np.array(P0), np.array(K), T, n, cfg)) - ref)
            for n in (20, 40, 80)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.8 < o < 4.3 for o in orders), (errs, orders)


def test_ode_update_touches_only_cells():
    st = np.array([[[Pm.EMPTY, Pm.PROLIF, Pm.QUIESC, Pm.DEAD, Pm.VESSEL, Pm.STROMA]]], dtype=np.uint8)
    cfg = Pm.Config(nx=6, ny=1, nz=1)
    phi = np.full(st.shape, 0.5)
    P = np.full(st.shape, 0.1)
    Vc = np.full(st.shape, 0.2)
    K = np.full(st.shape, 5.0)
    phi2, P2, V2 = ode_update(st, phi, P, Vc, K, cfg)
    moved_phi = phi2 != phi
    moved_P = P2 != P
    assert moved_phi.reshape(-1).tolist() == [False, True, True, False, False, False]
    assert moved_P.reshape(-1).tolist() == [False, True, True, False, False, True]
    assert (V2 != Vc).reshape(-1).tolist() == [False, True, True, False, False, True]
