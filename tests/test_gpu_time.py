"""Time discretisations on the GPU (drug_scheme / drug_substeps, o2_scheme /
o2_substeps: implicit Euler and Crank-Nicolson sub-steps, Section 2.4.1)
against the FP64 oracle (oracle.model.drug_step, o2_transient_step).

Tolerances: FP64 solves run to 1e-12 and are compared at 1e-9 relative (the
operator's conditioning times the tolerance, summed over the sub-steps);
FP32 storage with defect correction at 1e-6 relative."""

import numpy as np
import pytest

from gpu_helpers import make_pair, random_states
from oracle import params as Pm
from oracle.model import OracleSim, drug_step, o2_transient_step
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu

SHAPE = (24, 40, 56)
CASES = [("f64", hca.HCA_PC_JACOBI), ("f64", hca.HCA_PC_MG), ("f32", hca.HCA_PC_MG)]


@pytest.mark.parametrize("precision,pc", CASES)
@pytest.mark.parametrize("scheme,m,step", [(1, 1, 3), (1, 3, 21), (0, 4, 3)])
def test_drug_substeps_match_oracle(precision, pc, scheme, m, step, rng):
    rtol = 1e-12 if precision == "f64" else 1e-9
    sim, cfg, _ = make_pair(SHAPE, precision, seed=31, n_drugs=2, rtol_drug=rtol, picard_maxit=1,
                            drug_scheme=scheme, drug_substeps=m, preconditioner=pc, uptake_G=(0.0, 0.05, 0.0))
    st = random_states(SHAPE, rng)
    sim.set_states(st)
    sim.set_step(step)
    G_old = [(rng.random(SHAPE) * 0.5).astype(sim.dtype) for _ in range(2)]
    for d in range(2):
        sim.set_field(hca.FIELD_DRUG[d], G_old[d])
    sim.stage(hca.STAGE_DRUGS)
    got = [sim.field(hca.FIELD_DRUG[d]) for d in range(2)]
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    s = sim.stats()
    sim.close()
    exact = Pm.Config(**{**cfg.__dict__, "rtol_drug": 1e-13})
    tol = 1e-9 if precision == "f64" else 1e-6
    for d in range(2):
        ref, infos = drug_step(st, perf, G_old[d].astype(np.float64), step, exact, d)
        assert len(infos) == m
        assert np.max(np.abs(got[d] - ref)) <= tol * max(1.0, np.max(np.abs(ref))), d
        # at rtol 1e-12 the recomputed residual sits a few eps * cond(A) above the recursive one
        assert s["drug_rel_residual"][d] <= 5 * rtol


@pytest.mark.parametrize("precision,pc", CASES)
@pytest.mark.parametrize("scheme,m", [(1, 2), (2, 1), (2, 3)])
def test_transient_oxygen_matches_oracle(precision, pc, scheme, m, rng):
    """dt = 0.05 min, so that the mass term 2/h is of the size of the
    consumption coefficient and the time terms matter."""
    rtol = 1e-12 if precision == "f64" else 1e-9
    sim, cfg, _ = make_pair(SHAPE, precision, seed=32, n_drugs=0, rtol_o2=rtol, picard_maxit=1, dt=0.05,
                            o2_scheme=scheme, o2_substeps=m, preconditioner=pc)
    st = random_states(SHAPE, rng)
    st.reshape(-1)[0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, SHAPE).astype(sim.dtype)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, K_prev)
    sim.stage(hca.STAGE_O2)
    got = sim.field(hca.FIELD_O2)
    s = sim.stats()
    sim.close()
    exact = Pm.Config(**{**cfg.__dict__, "rtol_o2": 1e-13})
    ref, infos = o2_transient_step(st, K_prev.astype(np.float64), exact)
    assert len(infos) == m
    tol = 1e-9 if precision == "f64" else 1e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    assert s["o2_rel_residual"] <= 5 * rtol
    # the time terms are not negligible here: the quasi-steady solve differs
    qs, _ = o2_transient_step(st, K_prev.astype(np.float64), Pm.Config(**{**exact.__dict__, "dt": 1e12}))
    assert np.max(np.abs(ref - qs)) > 1e-3 * np.max(np.abs(ref))


def test_coupled_crank_nicolson_steps_match_oracle():
    n = 16
    params = dict(n_drugs=2, seed=33, rtol_o2=1e-13, rtol_drug=1e-13, picard_tol=1e-12,
                  drug_scheme=1, drug_substeps=2, o2_scheme=2, o2_substeps=2)
    maps = make_maps(n, n, n, corr_len=3.0, seed=33)
    sim = hca.Sim.create(n, n, n, maps.p_cell, maps.perf, maps.p_vessel, **params)
    orc = OracleSim(Pm.Config(nx=n, ny=n, nz=n, **params), maps.p_cell, maps.perf, maps.p_vessel)
    for step in range(3):
        sim.step(1)
        orc.step(1)
        assert np.array_equal(sim.states(), orc.state), f"states differ after step {step}"
        for bit, ref in ((hca.FIELD_O2, orc.K), (hca.FIELD_DRUG0, orc.G[0]), (hca.FIELD_DRUG1, orc.G[1])):
            got = sim.field(bit)
            assert np.max(np.abs(got - ref)) <= 1e-9 * max(1e-3, np.max(np.abs(ref))), (step, bit)
    sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_substep_graph_and_host_loop_agree_bitwise(precision, monkeypatch):
    shape = (24, 40, 56)
    out = []
    for no_graph in ("0", "1"):
        monkeypatch.setenv("HCA_NO_GRAPH", no_graph)
        sim, _, _ = make_pair(shape, precision, seed=34, n_drugs=2, preconditioner=hca.HCA_PC_MG,
                              drug_scheme=1, drug_substeps=3, o2_scheme=1, o2_substeps=2)
        sim.step(2)
        out.append((sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG[1]), sim.stats()))
        sim.close()
    (s0, K0, G0, st0), (s1, K1, G1, st1) = out
    assert np.array_equal(s0, s1) and np.array_equal(K0, K1) and np.array_equal(G0, G1)
    assert st0["drug_iterations"] == st1["drug_iterations"]


def test_batch_with_substeps_matches_single_runs():
    cfg_common = dict(n_drugs=1, drug_scheme=1, drug_substeps=2, o2_scheme=2, o2_substeps=2)
    sizes = [12, 20]
    cfgs, maps, single = [], [], []
    for r, n in enumerate(sizes):
        m = make_maps(n, n, n, corr_len=3.0, seed=40 + r)
        maps.append((m.p_cell, m.perf, m.p_vessel))
        cfgs.append(hca.make_config(n, n, n, seed=40 + r, **cfg_common))
        s = hca.Sim(cfgs[-1], maps[-1])
        s.step(2)
        single.append((s.states(), s.field(hca.FIELD_DRUG0), s.field(hca.FIELD_O2)))
        s.close()
    b = hca.Sim(cfgs, maps, batch=True)
    b.step(2)
    for r in range(2):
        assert np.array_equal(b.states(r), single[r][0])
        assert np.array_equal(b.field(hca.FIELD_DRUG0, r), single[r][1])
        assert np.array_equal(b.field(hca.FIELD_O2, r), single[r][2])
    b.close()


def test_time_scheme_config_errors():
    maps = make_maps(8, 8, 8, corr_len=1.0, seed=0)
    args = (8, 8, 8, maps.p_cell, maps.perf, maps.p_vessel)
    for bad in (dict(drug_scheme=2), dict(o2_scheme=3), dict(drug_substeps=0), dict(o2_substeps=0)):
        with pytest.raises(hca.HcaError) as e:
            hca.Sim.create(*args, **bad)
        assert e.value.status == hca.HCA_ERR_ARG, bad
    for bad in (dict(o2_scheme=1, o2_nonlinear=1), dict(o2_scheme=2, warm_start=hca.HCA_WS_LEARNED)):
        with pytest.raises(hca.HcaError) as e:
            hca.Sim.create(*args, **bad)
        assert e.value.status == hca.HCA_ERR_UNIMPLEMENTED, bad
    cfgs = [hca.make_config(8, 8, 8, drug_substeps=v) for v in (1, 2)]
    with pytest.raises(hca.HcaError) as e:
        hca.Sim(cfgs, [(maps.p_cell, maps.perf, maps.p_vessel)] * 2, batch=True)
    assert e.value.status == hca.HCA_ERR_ARG
