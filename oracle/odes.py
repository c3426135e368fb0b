"""Per-cell ODEs over one CA step with the oxygen K fixed at the cell's site.

Eq. (cellcycle):  dphi/dt = K / (T (K_phi + K))
Eq. (odep53):     dP/dt   = k1 - k1' K/(K_p53 + K) P
Eq. (odevegf):    dVc/dt  = k2 + k2'' P Vc/(J5 + Vc) - k2' K/(K_V + K) Vc

Section 2.4.2: the cell-cycle clock is integrated analytically, P has an
explicit solution over a step, and Vc was integrated with SciPy's VODE (Adams,
maximum step 1 min).  Here Vc uses classical fourth-order Runge-Kutta with a
fixed step h = dt / substeps (1 min by default), evaluating P exactly at each
stage time.

The phi update applies to cancer cells (PROLIF, QUIESC); P and Vc to every
cell (cancer and stroma).  Other sites are left unchanged.
"""

from __future__ import annotations

import numpy as np

from . import params as Pm


def phi_advance(phi, K, dt: float, cfg: Pm.Config):
    """Exact solution of Eq. (cellcycle) over dt at fixed K (linear in time)."""
    return phi + dt * K / (cfg.T_cycle * (cfg.K_phi + K))


def p53_rate(K, cfg: Pm.Config):
    """Degradation rate lambda = k1' K / (K_p53 + K) of Eq. (odep53)."""
    return cfg.k1p * K / (cfg.K_p53 + K)


def p53_at(P0, lam, s, cfg: Pm.Config):
    """Exact P(s) = P0 e^{-lam s} + k1 (1 - e^{-lam s}) / lam  (P0 + k1 s if lam = 0)."""
    lam = np.asarray(lam, dtype=np.float64)
    safe = np.where(lam != 0.0, lam, 1.0)
    decayed = P0 * np.exp(-lam * s) - cfg.k1 * np.expm1(-lam * s) / safe
    return np.where(lam != 0.0, decayed, P0 + cfg.k1 * s)


def vegf_rhs(Vc, Ps, K, cfg: Pm.Config):
    """Right-hand side of Eq. (odevegf) at fixed K and given P."""
    return cfg.k2 + cfg.k2pp * Ps * Vc / (cfg.J5 + Vc) - cfg.k2p * K / (cfg.K_V + K) * Vc


def vegf_rk4(Vc0, P0, K, dt: float, substeps: int, cfg: Pm.Config):
    """Classical RK4 for Vc with P(s) taken from its exact solution."""
    lam = p53_rate(K, cfg)
    h = dt / substeps
    V = np.array(Vc0, dtype=np.float64, copy=True)
    for m in range(substeps):
        s = m * h
        P_a = p53_at(P0, lam, s, cfg)
        P_b = p53_at(P0, lam, s + 0.5 * h, cfg)
        P_c = p53_at(P0, lam, s + h, cfg)
        k_1 = vegf_rhs(V, P_a, K, cfg)
        k_2 = vegf_rhs(V + 0.5 * h * k_1, P_b, K, cfg)
        k_3 = vegf_rhs(V + 0.5 * h * k_2, P_b, K, cfg)
        k_4 = vegf_rhs(V + h * k_3, P_c, K, cfg)
        V = V + (h / 6.0) * (k_1 + 2.0 * k_2 + 2.0 * k_3 + k_4)
    return V


def ode_update(state, phi, P, Vc, K, cfg: Pm.Config):
    """Advance phi, P, Vc of every cell by one CA step dt (returns new arrays)."""
    K = np.asarray(K, dtype=np.float64)
    cancer = np.isin(state, Pm.CANCER_STATES)
    cell = np.isin(state, Pm.CONSUMER_STATES)
    phi = np.asarray(phi, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    Vc = np.asarray(Vc, dtype=np.float64)
    phi_new = np.where(cancer, phi_advance(phi, K, cfg.dt, cfg), phi)
    lam = p53_rate(K, cfg)
    P_new = np.where(cell, p53_at(P, lam, cfg.dt, cfg), P)
    V_new = np.where(cell, vegf_rk4(Vc, P, K, cfg.dt, cfg.ode_substeps, cfg), Vc)
    return phi_new, P_new, V_new
