"""Plasma drug concentration G_{d,0}(t) after repeated bolus doses.

Eq. (intrachemo3): a one-compartment model dG/dt = -k G, reset to the dose
level at each administration time; the paper evaluates it in closed form
(Sections 2.2.3 and 2.4.2).  With boluses of peak level ``peak`` at
t_n = n * interval (n = 0, 1, 2, ...), the concentration is the sum of the
decaying contributions of all doses given so far:

    G_0(t) = sum_{n : t_n <= t} peak * exp(-k (t - t_n)).

Reading: the printed condition G(t_n) = d_n / V is taken as each bolus
raising the plasma level by d_n / V, so the closed forms of successive doses
superpose (the usual multiple-dose closed form).  A literal reset would
differ only by the previous dose's residue, which after 21 hourly steps is
below 1e-29 of the peak for epirubicin and about 13 % for cyclophosphamide.
"""

from __future__ import annotations

import math


def plasma_concentration(t: float, peak: float, decay: float, interval: float) -> float:
    """Closed form G_0(t) for boluses at 0, interval, 2*interval, ... (t >= 0)."""
    if t < 0:
        return 0.0
    total = 0.0
    n = 0
    while n * interval <= t:
        total += peak * math.exp(-decay * (t - n * interval))
        n += 1
        if interval <= 0:
            break
    return total
