"""The VEGF field and the vascular birth-death automaton (Sections 2.2.2 and
2.3, Eq. vac_v and Eq. vascular_module), without Avastin.

VEGF: with A = 0 Eq. (vac_v) is linear, dV/dt = D_V lap V + a_V Vc [cell]
- psi_V V, cells being the consuming states (cancer and stroma) and Vc their
intracellular VEGF.  It is stepped like the drugs (implicit Euler or
Crank-Nicolson sub-steps, oracle.model.vegf_step).

Vascular update, every vessel_interval steps after the cell update (Algorithm
1 updates G with L), one Philox draw u per site keyed (seed, site, step,
VASCULAR):
  * a vessel with V < V_low or V > V_high is removed (site EMPTY) if u < p_death;
  * a free site (EMPTY or DEAD) with V_low <= V <= V_high becomes a vessel if
    u < p_birth(x), where
        p_birth(x) = min(1, E[n_new] V(x) / sum_candidates V),
        E[n_new]   = beta_birth * sum_vessels V / (V_sprout + V),
    so the expected number of new vessels follows the E[n_new] formula of
    Section 2.2.2 (its constants lumped in beta_birth) and the birth
    probability is proportional to V, as the text states.
Readings: the two sums are taken in 2^-32 fixed point (per-site terms
floor(x 2^32) of x = V/(V_sprout + V) and of x = V/V_high, summed exactly as
integers), so their value does not depend on summation order; the ratio is
then evaluated in FP64 as (beta * S1 * (V / V_high)) / S2.  A vessel site's
perfusion keeps its map value.  Test infrastructure only.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import params as Pm
from .philox import site_uniform

FIX = float(2 ** 32)


@dataclasses.dataclass
class VascularStats:
    births: int = 0
    deaths: int = 0


def fixed_sum(x) -> int:
    """Exact integer sum of floor(x * 2^32) over the given values (x >= 0)."""
    q = np.floor(np.asarray(x, dtype=np.float64) * FIX).astype(np.int64)
    return int(q.sum(dtype=np.int64))


def vascular_update(state, V, cfg: Pm.Config, step: int):
    st = np.array(state, dtype=np.uint8, copy=True).reshape(-1)
    dtype = np.float32 if cfg.precision == "f32" else np.float64
    Vf = np.asarray(V, dtype=dtype).astype(np.float64).reshape(-1)
    in_range = (Vf >= cfg.V_low) & (Vf <= cfg.V_high)
    vessel = st == Pm.VESSEL
    cand = np.isin(st, Pm.FREE_STATES) & in_range
    S1 = fixed_sum(Vf[vessel] / (cfg.V_sprout + Vf[vessel]))
    S2 = fixed_sum(Vf[cand] / cfg.V_high)
    u = site_uniform(cfg.seed, np.arange(st.size, dtype=np.uint64), step, Pm.PURPOSE_VASCULAR)
    stats = VascularStats()
    for i in np.flatnonzero(vessel & ~in_range):
        if u[i] < cfg.p_death:
            st[i] = Pm.EMPTY
            stats.deaths += 1
    if S2 > 0:
        for i in np.flatnonzero(cand):
            p = min(1.0, (cfg.beta_birth * float(S1) * (Vf[i] / cfg.V_high)) / float(S2))
            if u[i] < p:
                st[i] = Pm.VESSEL
                stats.births += 1
    return st.reshape(state.shape), stats
