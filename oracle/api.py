"""The oracle behind the library's call names: oracle_create, oracle_step,
oracle_read_fields, oracle_read_states, oracle_get_stats, oracle_destroy
(FP64 only), so that a test can drive both sides with the same sequence of
calls.  Test infrastructure only; a thin veneer over oracle.model.OracleSim.

Field bits are those of the library (O2 1, DRUG0..2 2/4/8, PHI 16, P53 32,
VEGFC 64, PERF 128, VEGF 256); fields come back packed in increasing bit
order, each in site order x + nx*(y + ny*z).
"""

from __future__ import annotations

import numpy as np

from . import params as Pm
from .model import OracleSim

FIELD_O2, FIELD_PHI, FIELD_P53, FIELD_VEGFC, FIELD_PERF, FIELD_VEGF = 1, 16, 32, 64, 128, 256
FIELD_DRUG = (2, 4, 8)


class OracleHandle:
    """One or more independent replicates (a batch is a list of simulations)."""

    def __init__(self, sims):
        self.sims = list(sims)


def oracle_create(cfg: Pm.Config, p_cell, perf, p_vessel) -> OracleHandle:
    return OracleHandle([OracleSim(cfg, p_cell, perf, p_vessel)])


def oracle_create_batch(cfgs, p_cells, perfs, p_vessels) -> OracleHandle:
    return OracleHandle([OracleSim(c, a, b, v) for c, a, b, v in zip(cfgs, p_cells, perfs, p_vessels)])


def oracle_step(h: OracleHandle, n_steps: int = 1) -> None:
    for s in h.sims:
        s.step(n_steps)


def _field(sim: OracleSim, bit: int) -> np.ndarray:
    if bit == FIELD_O2:
        return sim.K
    if bit in FIELD_DRUG:
        d = FIELD_DRUG.index(bit)
        if d >= sim.cfg.n_drugs:
            raise ValueError("no such drug")
        return sim.G[d]
    if bit == FIELD_VEGF:
        if not sim.cfg.vegf:
            raise ValueError("no VEGF field")
        return sim.V
    return {FIELD_PHI: sim.phi, FIELD_P53: sim.P, FIELD_VEGFC: sim.Vc, FIELD_PERF: sim.perf}[bit]


def oracle_read_fields(h: OracleHandle, rep: int, mask: int) -> np.ndarray:
    sim = h.sims[rep]
    bits = [1 << k for k in range(9) if mask & (1 << k)]
    if not bits or mask & ~0x1FF:
        raise ValueError("bad field mask")
    return np.concatenate([np.asarray(_field(sim, b), dtype=np.float64).reshape(-1) for b in bits])


def oracle_read_states(h: OracleHandle, rep: int) -> np.ndarray:
    return h.sims[rep].state.reshape(-1).copy()


def oracle_get_stats(h: OracleHandle, rep: int) -> dict:
    sim = h.sims[rep]
    out = {"step": sim.step_index, "picard_iterations": sim.picard_iterations}
    if sim.history:
        last = sim.history[-1]
        out.update(committed=last.committed, kills=last.kills, divisions=last.divisions, blocked=last.blocked,
                   counts=[int(c) for c in last.counts], vessel_births=last.vessel_births,
                   vessel_deaths=last.vessel_deaths)
        if last.o2 is not None:
            out.update(o2_iterations=last.o2.iterations, o2_rel_residual=last.o2.rel_residual)
        out["drug_iterations"] = [i.iterations for i in last.drugs]
    return out


def oracle_destroy(h: OracleHandle) -> None:
    h.sims.clear()
