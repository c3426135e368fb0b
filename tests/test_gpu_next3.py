"""The VEGF field (Eq. vac_v with A = 0), the vascular birth-death automaton
and the Michaelis-Menten / three-compartment plasma models on the GPU against
the FP64 oracle (oracle.model.vegf_step, oracle.vascular, oracle.pk).

Tolerances: fields 1e-9 relative (FP64, solves at 1e-12) and 1e-6 (FP32 with
defect correction); vascular and cell states bit-exact (the vascular sums are
exact integers on both sides)."""

import numpy as np
import pytest

from gpu_helpers import make_pair, random_states
from oracle import params as Pm
from oracle.ca import ca_update
from oracle.model import OracleSim, drug_step, vegf_step
from oracle.vascular import vascular_update
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu

SHAPE = (20, 28, 44)
CASES = [("f64", hca.HCA_PC_JACOBI), ("f64", hca.HCA_PC_MG), ("f32", hca.HCA_PC_MG)]


@pytest.mark.parametrize("precision,pc", CASES)
@pytest.mark.parametrize("scheme,m", [(0, 1), (1, 3)])
def test_vegf_solve_matches_oracle(precision, pc, scheme, m, rng):
    rtol = 1e-12 if precision == "f64" else 1e-9
    sim, cfg, _ = make_pair(SHAPE, precision, seed=81, n_drugs=0, vegf=1, rtol_drug=rtol, picard_maxit=1,
                            drug_scheme=scheme, drug_substeps=m, preconditioner=pc)
    st = random_states(SHAPE, rng)
    sim.set_states(st)
    Vc = rng.random(SHAPE).astype(sim.dtype)
    V0 = (rng.random(SHAPE) * 1e-4).astype(sim.dtype)
    sim.set_field(hca.FIELD_VEGFC, Vc)
    sim.set_field(hca.FIELD_VEGF, V0)
    sim.stage(hca.STAGE_O2)
    got = sim.field(hca.FIELD_VEGF)
    s = sim.stats()
    sim.close()
    exact = Pm.Config(**{**cfg.__dict__, "rtol_drug": 1e-14})
    ref, infos = vegf_step(st, V0.astype(np.float64), Vc.astype(np.float64), exact)
    tol = 1e-9 if precision == "f64" else 1e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    # the recomputed FP64 residual floors near eps * cond(A) ~ 3e-12 for this operator
    assert s["vegf_rel_residual"] <= 10 * rtol and s["vegf_iterations"] > 0


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(6, 7, 13), (17, 23, 31)])
def test_vascular_update_bit_exact(shape, precision, rng):
    for trial in range(3):
        step = 11 + 12 * trial
        sim, cfg, _ = make_pair(shape, precision, seed=82 + trial, n_drugs=1, vegf=1, vessel_interval=12,
                                picard_maxit=1, p_death=0.4, beta_birth=3.0, V_high=2e-3)
        st = rng.choice([Pm.EMPTY, Pm.PROLIF, Pm.DEAD, Pm.VESSEL, Pm.STROMA], size=shape,
                        p=[0.4, 0.3, 0.05, 0.15, 0.1]).astype(np.uint8)
        V = (10 ** rng.uniform(-7, -2.4, shape)).astype(sim.dtype)
        sim.set_states(st)
        sim.set_field(hca.FIELD_VEGF, V)
        sim.set_field(hca.FIELD_PHI, np.zeros(shape))      # no cell commits: only DEAD -> EMPTY
        sim.set_step(step)
        sim.stage(hca.STAGE_CA)
        st1, *_ = ca_update(st, np.zeros(shape), np.zeros(shape), np.zeros(shape), np.zeros(shape),
                            [np.zeros(shape)], cfg, step)
        ref, vs = vascular_update(st1, V.astype(np.float64), cfg, step)
        assert np.array_equal(sim.states(), ref)
        s = sim.stats()
        assert (s["vessel_births"], s["vessel_deaths"]) == (vs.births, vs.deaths)
        assert vs.births > 0 and vs.deaths > 0
        # not a vascular step: nothing changes
        sim.set_states(st)
        sim.set_step(step + 1)
        sim.stage(hca.STAGE_CA)
        assert np.array_equal(sim.states(), st1)
        sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("step", [3, 21, 40])
def test_pk_models_match_oracle(precision, step, rng):
    rtol = 1e-12 if precision == "f64" else 1e-9
    sim, cfg, _ = make_pair(SHAPE, precision, seed=83, n_drugs=3, rtol_drug=rtol, picard_maxit=1,
                            pk_model=(0, 2, 1), dose_peak=(1.0, 1.0, 54.0), drug_scheme=1, drug_substeps=2)
    st = random_states(SHAPE, rng)
    sim.set_states(st)
    sim.set_step(step)
    G_old = [(rng.random(SHAPE) * 0.5).astype(sim.dtype) for _ in range(3)]
    for d in range(3):
        sim.set_field(hca.FIELD_DRUG[d], G_old[d])
    sim.stage(hca.STAGE_DRUGS)
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    got = [sim.field(hca.FIELD_DRUG[d]) for d in range(3)]
    sim.close()
    exact = Pm.Config(**{**cfg.__dict__, "rtol_drug": 1e-14})
    tol = 1e-9 if precision == "f64" else 1e-6
    for d in range(3):
        ref, _ = drug_step(st, perf, G_old[d].astype(np.float64), step, exact, d)
        assert np.max(np.abs(got[d] - ref)) <= tol * max(1.0, np.max(np.abs(ref))), d


def test_coupled_run_matches_oracle():
    n = 16
    params = dict(n_drugs=3, seed=84, rtol_o2=1e-13, rtol_drug=1e-13, picard_tol=1e-12, vegf=1, vessel_interval=2,
                  pk_model=(0, 2, 1), V_high=5e-5, beta_birth=0.5, p_death=0.5)
    maps = make_maps(n, n, n, corr_len=3.0, seed=84)
    sim = hca.Sim.create(n, n, n, maps.p_cell, maps.perf, maps.p_vessel, **params)
    orc = OracleSim(Pm.Config(nx=n, ny=n, nz=n, **params), maps.p_cell, maps.perf, maps.p_vessel)
    events = 0
    for step in range(5):
        sim.step(1)
        orc.step(1)
        assert np.array_equal(sim.states(), orc.state), f"states differ after step {step}"
        for bit, ref in ((hca.FIELD_O2, orc.K), (hca.FIELD_VEGF, orc.V), (hca.FIELD_DRUG[2], orc.G[2]),
                         (hca.FIELD_DRUG[1], orc.G[1])):
            got = sim.field(bit)
            assert np.max(np.abs(got - ref)) <= 1e-9 * max(1e-12, np.max(np.abs(ref))), (step, bit)
        s, h = sim.stats(), orc.history[-1]
        assert (s["vessel_births"], s["vessel_deaths"]) == (h.vessel_births, h.vessel_deaths)
        events += h.vessel_births + h.vessel_deaths
    assert events > 0
    sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_graph_and_host_loop_agree_bitwise(precision, monkeypatch):
    out = []
    for no_graph in ("0", "1"):
        monkeypatch.setenv("HCA_NO_GRAPH", no_graph)
        sim, _, _ = make_pair((24, 40, 56), precision, seed=85, n_drugs=2, preconditioner=hca.HCA_PC_MG, vegf=1,
                              vessel_interval=1, V_high=5e-5, beta_birth=0.5, pk_model=(0, 2, 1))
        sim.step(3)
        out.append((sim.states(), sim.field(hca.FIELD_VEGF), sim.field(hca.FIELD_DRUG[1]), sim.stats()))
        sim.close()
    (s0, V0, G0, st0), (s1, V1, G1, st1) = out
    assert np.array_equal(s0, s1) and np.array_equal(V0, V1) and np.array_equal(G0, G1)
    assert st0["vegf_iterations"] == st1["vegf_iterations"]


def test_next3_config_errors():
    maps = make_maps(8, 8, 8, corr_len=1.0, seed=0)
    args = (8, 8, 8, maps.p_cell, maps.perf, maps.p_vessel)
    for bad in (dict(vegf=2), dict(vessel_interval=3), dict(vegf=1, vessel_interval=-1),
                dict(vegf=1, vessel_interval=2, V_high=0.0), dict(pk_model=(3, 0, 0)),
                dict(n_drugs=1, pk_model=(1, 0, 0), mm_km=0.0)):
        with pytest.raises(hca.HcaError) as e:
            hca.Sim.create(*args, **bad)
        assert e.value.status == hca.HCA_ERR_ARG, bad
    sim = hca.Sim.create(*args)
    with pytest.raises(hca.HcaError):
        sim.field(hca.FIELD_VEGF)          # no VEGF field without vegf = 1
    sim.close()
