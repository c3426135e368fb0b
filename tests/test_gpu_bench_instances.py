"""Parity of the kernel instances the 256^3 bench runs.

The bench lattice has 64 four-site groups per row, so every row-kernel runs
with two groups per lane (the compile-time NI = 2 instances); they are used
for any row of 129..256 sites.  Here the FP32 + multigrid + defect-correction
solves of oxygen and two drugs on such lattices (autotuned launch shape, as in
the bench) are compared element by element with the FP64 oracle's solves of
the same systems (Eqs. oxygen and chemo, Section 2.4.1), and at the full
256^3 bench workload the FP64 residual of the stored two-word fields
(hi + lo) is recomputed on the host with the oracle's stencil:

* field tolerance: 1e-6 of the field's maximum (FP32 storage);
* residual at 256^3: the FP64 relative residual of hi + lo for the system the
  library solves (its FP32 coefficients, rebuilt here in numpy float32 with
  the same operations) must meet the solve tolerance rtol = 1e-8 (the
  library's own stopping test is float-float, ~48 bits), and for the oracle's
  FP64 coefficients it stays within the FP32 rounding of those coefficients
  (1e-6).
"""

import numpy as np
import pytest

from gpu_helpers import make_pair, random_states
from oracle import multigrid as MG
from oracle import params as Pm
from oracle import stencil as S
from oracle.model import plasma_levels
from paper_2105_00448_gb300 import hca

pytestmark = pytest.mark.gpu

# (nz, ny, nx): rows of 160, 256 and 130 sites (40, 64, 33 groups: two per lane)
SHAPES = [(24, 32, 160), (16, 16, 256), (13, 21, 130)]


def groups_per_lane(nx):
    gpr = (nx + 3) // 4
    lpr = min(32, 1 << (gpr - 1).bit_length())
    return (gpr + lpr - 1) // lpr


def two_word(sim, hi_bit, lo_bit):
    return sim.field(hi_bit).astype(np.float64) + sim.field(lo_bit).astype(np.float64)


@pytest.mark.parametrize("shape", SHAPES)
def test_ni2_fp32_mg_solves_match_oracle(shape):
    assert groups_per_lane(shape[2]) == 2
    rng = np.random.default_rng(40 + shape[2])
    sim, cfg, _ = make_pair(shape, "f32", seed=6, n_drugs=2, rtol_o2=1e-8, rtol_drug=1e-8, picard_maxit=1,
                            preconditioner=hca.HCA_PC_MG)
    st = random_states(shape, rng)
    st.reshape(-1)[0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, shape).astype(np.float32)
    G_old = [(rng.random(shape) * 0.5).astype(np.float32) for _ in range(2)]
    sim.set_states(st)
    sim.set_step(3)
    sim.set_field(hca.FIELD_O2, K_prev)
    for d in range(2):
        sim.set_field(hca.FIELD_DRUG[d], G_old[d])
    sim.stage(hca.STAGE_O2 | hca.STAGE_DRUGS)
    K = sim.field(hca.FIELD_O2)
    G = [sim.field(hca.FIELD_DRUG[d]) for d in range(2)]
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    s = sim.stats()
    sim.close()
    assert s["o2_rel_residual"] <= 1e-8 and max(s["drug_rel_residual"][:2]) <= 1e-8
    cK, aK = S.o2_coupling(cfg), S.o2_reaction(st, K_prev.astype(np.float64), cfg)
    refK, _ = MG.mg_pcg(cK, aK, S.o2_rhs(st, cfg), K_prev.astype(np.float64), 1e-12, 1000)
    assert np.max(np.abs(K - refK)) <= 1e-6 * np.max(np.abs(refK))
    G0 = plasma_levels(cfg, 4 * cfg.dt)
    for d in range(2):
        cG, aG = S.drug_coupling(cfg, d), S.drug_reaction(st, perf, cfg, d)
        b = S.drug_rhs(st, perf, G_old[d].astype(np.float64), G0[d], cfg, d)
        refG, _ = MG.mg_pcg(cG, aG, b, G_old[d].astype(np.float64), 1e-12, 1000)
        assert np.max(np.abs(G[d] - refG)) <= 1e-6 * max(1.0, np.max(np.abs(refG)))


def _rel_residual(b, coupling, reaction, x):
    r = b - S.apply_operator(x, coupling, reaction)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def test_fullsize_fp64_residual_of_two_word_fields():
    """The 256^3 bench workload: after two warm-up steps, one oxygen and drug
    stage; the FP64 residuals of hi + lo on the host."""
    import bench
    from synth import make_maps

    n = bench.N_EDGE
    maps = make_maps(n, n, n, corr_len=bench.CORR_LEN, seed=bench.WORKLOAD["seed"])
    cfg_h = hca.make_config(n, n, n, **bench.WORKLOAD)
    sim = hca.Sim(cfg_h, (maps.p_cell, maps.perf, maps.p_vessel))
    sim.step(2, allow_noconv=True)
    st = sim.states()
    step = 2
    K_prev_hi, K_prev_lo = sim.field(hca.FIELD_O2), sim.field(hca.FIELD_O2_LO)
    G_old = [two_word(sim, hca.FIELD_DRUG[d], hca.FIELD_DRUG0_LO << d) for d in range(2)]
    perf32 = sim.field(hca.FIELD_PERF)
    sim.stage(hca.STAGE_O2 | hca.STAGE_DRUGS)
    K = two_word(sim, hca.FIELD_O2, hca.FIELD_O2_LO)
    G = [two_word(sim, hca.FIELD_DRUG[d], hca.FIELD_DRUG0_LO << d) for d in range(2)]
    s = sim.stats()
    sim.close()
    params = {k: v for k, v in bench.WORKLOAD.items() if k in Pm.Config.__dataclass_fields__}
    cfg = Pm.Config(nx=n, ny=n, nz=n, **params)
    f32 = np.float32
    vessel = st == Pm.VESSEL
    consumer = np.isin(st, Pm.CONSUMER_STATES)
    cancer = np.isin(st, Pm.CANCER_STATES)

    # oxygen, the library's FP32 system: a = phi_K / (K1 + K_prev) at consumers
    # (K_prev = hi + lo rounded to FP32), + r_K at vessels; b = r_K K0 at vessels
    lag = K_prev_hi + K_prev_lo                                  # float32 sum
    a32 = np.where(consumer, f32(cfg.phi_K) / (f32(cfg.K1) + lag), f32(0))
    a32 = np.where(vessel, a32 + f32(cfg.r_K), a32).astype(np.float64)
    b32 = np.where(vessel, f32(cfg.r_K * cfg.K0), f32(0)).astype(np.float64)
    c32 = float(f32(S.o2_coupling(cfg)))
    rel = _rel_residual(b32, c32, a32, K)
    assert rel <= 1e-8 * (1 + 1e-3), rel
    assert abs(rel - s["o2_rel_residual"]) <= 1e-3 * rel + 1e-12
    # the oracle's FP64 coefficients at the same K_prev
    rel64 = _rel_residual(S.o2_rhs(st, cfg), S.o2_coupling(cfg), S.o2_reaction(st, lag.astype(np.float64), cfg), K)
    assert rel64 <= 1e-6, rel64

    # drugs: a = (1/dt + psi) + kappa perf at vessels (+ uptake at cancer
    # sites); b = (G_old / dt) rounded to FP32 + kappa perf G_0(t^{n+1}) at vessels
    G0 = plasma_levels(cfg, (step + 1) * cfg.dt)
    for d in range(2):
        base = f32(1.0 / cfg.dt + cfg.psi_G[d])
        a = np.where(vessel, base + f32(cfg.kappa_G[d]) * perf32, base)
        a = np.where(cancer, a + f32(cfg.uptake_G[d]), a).astype(np.float64)
        src = np.where(vessel, f32(cfg.kappa_G[d]) * perf32 * f32(G0[d]), f32(0))
        b = ((G_old[d] / cfg.dt).astype(np.float32) + src).astype(np.float64)
        c = float(f32(S.drug_coupling(cfg, d)))
        rel = _rel_residual(b, c, a, G[d])
        assert rel <= 1e-8 * (1 + 1e-3), (d, rel)
        assert abs(rel - s["drug_rel_residual"][d]) <= 1e-3 * rel + 1e-12
        perf = perf32.astype(np.float64)
        rel64 = _rel_residual(S.drug_rhs(st, perf, G_old[d], G0[d], cfg, d), S.drug_coupling(cfg, d),
                              S.drug_reaction(st, perf, cfg, d), G[d])
        assert rel64 <= 1e-6, (d, rel64)
