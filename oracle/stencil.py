"""Discrete operators of the oxygen and drug reaction-diffusion equations.

The paper discretises Eq. (oxygen) and Eq. (chemo) with P1 finite elements on
refined meshes (Section 2.4.1).  Here they are discretised on the CA lattice
itself with the standard 7-point finite-difference Laplacian, one unknown per
site, and homogeneous Neumann boundaries (a neighbour outside the box is
omitted, so each row of the Laplacian sums to zero).  The delta-function
source and sink sums N_c, N_v (Eq. delta_function) become per-site indicators
of the site's state.

Arrays are float64 with shape (nz, ny, nx); site index x + nx*(y + ny*z).
"""

from __future__ import annotations

import numpy as np

from . import params as P


def laplacian_sum(u: np.ndarray) -> np.ndarray:
    """S(u)_i = sum over in-box face neighbours j of (u_i - u_j)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    for axis in range(u.ndim):
        d = np.diff(u, axis=axis)                     # u[k+1] - u[k]
        lo = [slice(None)] * u.ndim
        hi = [slice(None)] * u.ndim
        lo[axis] = slice(0, -1)
        hi[axis] = slice(1, None)
        out[tuple(lo)] -= d                           # site k:   u_k - u_{k+1}
        out[tuple(hi)] += d                           # site k+1: u_{k+1} - u_k
    return out


def neighbour_count(shape) -> np.ndarray:
    """Number of in-box face neighbours of every site (3 .. 6 in 3-D)."""
    n = np.zeros(shape, dtype=np.float64)
    for axis, extent in enumerate(shape):
        c = np.full(extent, 2.0)
        if extent >= 1:
            c[0] -= 1.0
            c[-1] -= 1.0
        view = [1] * len(shape)
        view[axis] = extent
        n += c.reshape(view)
    return n


def apply_operator(u: np.ndarray, coupling: float, reaction: np.ndarray) -> np.ndarray:
    """A u = coupling * S(u) + reaction * u  (coupling = D / dx^2)."""
    return coupling * laplacian_sum(u) + reaction * u


def jacobi_diagonal(shape, coupling: float, reaction: np.ndarray) -> np.ndarray:
    """Diagonal of A: coupling * (number of neighbours) + reaction."""
    return coupling * neighbour_count(shape) + reaction


def is_consumer(state):
    return np.isin(state, P.CONSUMER_STATES)


def is_vessel(state):
    return state == P.VESSEL


def is_live_cancer(state):
    return np.isin(state, P.CANCER_STATES)


# ---------------------------------------------------------------- oxygen ---
def o2_coupling(cfg: P.Config) -> float:
    return cfg.D_K / cfg.dx ** 2


def o2_reaction(state, K_prev, cfg: P.Config) -> np.ndarray:
    """Lagged-linearised reaction coefficient of Eq. (oxygen) with s_K = 0.

    Consumption phi_K K/(K1 + K) at consuming sites is linearised as
    phi_K K/(K1 + K_prev) (Section 2.4.1, linear approximation); vessel sites
    add the supply coefficient r_K.
    """
    K_prev = np.asarray(K_prev, dtype=np.float64)
    cons = np.where(is_consumer(state), cfg.phi_K / (cfg.K1 + K_prev), 0.0)
    return cons + np.where(is_vessel(state), cfg.r_K, 0.0)


def o2_rhs(state, cfg: P.Config) -> np.ndarray:
    """Right-hand side r_K K0 at vessel sites (the source term of Eq. oxygen)."""
    return np.where(is_vessel(state), cfg.r_K * cfg.K0, 0.0)


# ------------------------------------------------- time discretisation ---
# With the spatial operator A_0 u = coupling S(u) + a u and source f, the
# semi-discrete equation du/dt = -A_0 u + f (s = 1 in Eq. oxygen, Eq. chemo)
# over a sub-step h becomes
#   implicit Euler:   (1/h + A_0) u^k = u^{k-1}/h + f^k
#   Crank-Nicolson:   (2/h + A_0) u^k = (2/h - A_0) u^{k-1} + f^{k-1} + f^k
# (the Crank-Nicolson form is the average of the two time levels, times 2).
def time_mass(scheme: int, h: float) -> float:
    """Coefficient added to the reaction: 1/h (implicit Euler), 2/h
    (Crank-Nicolson)."""
    return {1: 1.0 / h, 2: 2.0 / h}[scheme]


def time_rhs(scheme: int, h: float, u_old, coupling: float, reaction0, f_old, f_new) -> np.ndarray:
    """Right-hand side of one sub-step; reaction0 is a of A_0 (no mass term)."""
    u_old = np.asarray(u_old, dtype=np.float64)
    if scheme == 1:
        return u_old / h + f_new
    return 2.0 * u_old / h - apply_operator(u_old, coupling, reaction0) + f_old + f_new


# ----------------------------------------------------------------- drugs ---
def drug_coupling(cfg: P.Config, d: int) -> float:
    return cfg.D_G[d] / cfg.dx ** 2


def drug_kappa(state, perf, cfg: P.Config, d: int) -> np.ndarray:
    """Vessel exchange coefficient kappa_i = kappa_G * perf_i at vessel sites.

    The paper's c_G K_trans S_MRI / (dx^2 N_v) * r_x/r0 (Eq. chemo) is a
    per-site permeability scale; the perfusion map stands in for K_trans and
    r_x/r0, and kappa_G collects the unpublished constants.
    """
    perf = np.asarray(perf, dtype=np.float64)
    return np.where(is_vessel(state), cfg.kappa_G[d] * perf, 0.0)


def drug_reaction0(state, perf, cfg: P.Config, d: int) -> np.ndarray:
    """Reaction of the spatial operator: psi + kappa_i [+ uptake at live cancer sites]."""
    kappa = drug_kappa(state, perf, cfg, d)
    uptake = np.where(is_live_cancer(state), cfg.uptake_G[d], 0.0)
    return cfg.psi_G[d] + kappa + uptake


def drug_reaction(state, perf, cfg: P.Config, d: int, mass=None) -> np.ndarray:
    """Reaction of the solved operator: mass + psi + kappa_i [+ uptake at live
    cancer sites], mass = 1/dt (one implicit-Euler step) unless given."""
    kappa = drug_kappa(state, perf, cfg, d)
    uptake = np.where(is_live_cancer(state), cfg.uptake_G[d], 0.0)
    m = 1.0 / cfg.dt if mass is None else mass
    return m + cfg.psi_G[d] + kappa + uptake


def drug_rhs(state, perf, G_old, G0_next: float, cfg: P.Config, d: int) -> np.ndarray:
    """G^n / dt + kappa_i G_{d,0}(t^{n+1})."""
    kappa = drug_kappa(state, perf, cfg, d)
    return np.asarray(G_old, dtype=np.float64) / cfg.dt + kappa * G0_next
