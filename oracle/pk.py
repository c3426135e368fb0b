"""Plasma drug levels G_{d,0}(t) for the three pharmacokinetic models of the
intravascular module (Section 2.2.3), with boluses of size ``peak`` (the
plasma level a dose adds) at t_n = n * interval, n = 0, 1, 2, ...

  0: one compartment, dG/dt = -k G: closed form, doses superposed
     (oracle.plasma.plasma_concentration);
  1: Michaelis-Menten (fluorouracil), dG/dt = -v_max G / (k_m + G): between
     doses G(t) = k_m W((G_s / k_m) exp((G_s - v_max (t - t_s)) / k_m)), W the
     principal Lambert W function, and each dose adds ``peak`` to the level
     just before it (the model is nonlinear, so doses do not superpose);
  2: three compartments (epirubicin), linear: the plasma level after a unit
     bolus is [exp(M t)]_00 with the rate matrix M of the compartment amounts,
       M = [[-(cl2 + q2 + q3)/w1, q2/w2, q3/w3],
            [ q2/w1,             -q2/w2, 0    ],
            [ q3/w1,              0,    -q3/w3]],
     and doses superpose.

Reading (model 2): the printed plasma equation has G_{2,1} and G_{2,2} in its
two loss terms; with them read as G_{2,0} the system conserves the drug
between compartments (the peripheral equations as printed are kept).
Test infrastructure only.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm
from scipy.special import lambertw

from . import params as Pm
from .plasma import plasma_concentration


def mm_decay(G_s: float, s: float, vmax: float, km: float) -> float:
    """Michaelis-Menten level a time s after the level G_s."""
    if G_s <= 0.0:
        return 0.0
    arg = (G_s / km) * math.exp((G_s - vmax * s) / km)
    return float(km * lambertw(arg, 0).real)


def plasma_mm(t: float, peak: float, vmax: float, km: float, interval: float) -> float:
    if t < 0:
        return 0.0
    G, t_prev, n = 0.0, 0.0, 0
    while n * interval <= t:
        t_n = n * interval
        G = mm_decay(G, t_n - t_prev, vmax, km) + peak if n > 0 else peak
        t_prev = t_n
        n += 1
        if interval <= 0:
            break
    return mm_decay(G, t - t_prev, vmax, km)


def three_compartment_matrix(cfg: Pm.Config) -> np.ndarray:
    w1, w2, w3 = cfg.epi_w
    q2, q3, cl2 = cfg.epi_q2, cfg.epi_q3, cfg.epi_cl2
    return np.array([[-(cl2 + q2 + q3) / w1, q2 / w2, q3 / w3],
                     [q2 / w1, -q2 / w2, 0.0],
                     [q3 / w1, 0.0, -q3 / w3]])


def plasma_three(t: float, peak: float, cfg: Pm.Config, interval: float) -> float:
    if t < 0:
        return 0.0
    M = three_compartment_matrix(cfg)
    total, n = 0.0, 0
    while n * interval <= t:
        total += peak * float(expm(M * (t - n * interval))[0, 0])
        n += 1
        if interval <= 0:
            break
    return total


def plasma_level(cfg: Pm.Config, d: int, t: float) -> float:
    """G_{d,0}(t) of drug d under its configured model."""
    period = cfg.dose_interval * cfg.dt
    model = cfg.pk_model[d]
    if model == 1:
        return plasma_mm(t, cfg.dose_peak[d], cfg.mm_vmax, cfg.mm_km, period)
    if model == 2:
        return plasma_three(t, cfg.dose_peak[d], cfg, period)
    return plasma_concentration(t, cfg.dose_peak[d], cfg.plasma_decay[d], period)
