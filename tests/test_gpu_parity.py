"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (the bars of the method's specification):
* integer and index work (Philox draws, seeding, CA states and counts): bit-exact;
* single operator applications and ODE updates on identical inputs:
  1e-12 relative (FP64 storage), 1e-6 relative (FP32 storage), relative to
  the size of the terms;
* solves run to a tight tolerance: compared at the level the tolerance and
  the operator's conditioning allow (stated per test).
Lattices are ragged (nx not a multiple of 4, rows not a multiple of the
32-row chunk) and span several chunks.
"""

import numpy as np
import pytest

from gpu_helpers import make_pair, operator_scale, random_states
from oracle import params as Pm
from oracle import stencil as S
from oracle.ca import ca_update
from oracle.model import OracleSim, drug_solve, o2_solve, seed_lattice
from oracle.odes import ode_update
from oracle.philox import site_uniform
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu

SHAPES = [(5, 7, 13), (11, 29, 37), (40, 48, 64), (3, 3, 1), (1, 1, 6)]
TOL = {"f64": 1e-12, "f32": 1e-6}


def test_philox_bit_identical_to_oracle():
    n = 1_000_000
    for seed, step, purpose, site0 in [(0, 0, 0, 0), (2**40 + 7, 13, 3, 5_000_000), (123456789, 2**31 + 5, 2, 2**33)]:
        gpu = hca.hca_philox_uniforms(seed, site0, n, step, purpose)
        ref = site_uniform(seed, np.arange(site0, site0 + n, dtype=np.uint64), step, purpose)
        assert np.array_equal(gpu.astype(np.float64), ref)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES[:3])
def test_seeding_bit_exact(shape, precision):
    sim, cfg, maps = make_pair(shape, precision, seed=11, n_drugs=1)
    st, phi = seed_lattice(cfg, maps.p_cell, maps.p_vessel)
    assert np.array_equal(sim.states(), st)
    assert np.array_equal(sim.field(hca.FIELD_PHI).astype(np.float64), phi)
    assert np.array_equal(sim.field(hca.FIELD_PERF), maps.perf.astype(sim.dtype))
    sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_operator_matches_oracle_stencil(shape, precision, rng):
    sim, cfg, maps = make_pair(shape, precision, seed=2, n_drugs=3, uptake_G=(0.0, 0.2, 0.0),
                               picard_maxit=1)
    st = random_states(shape, rng)
    sim.set_states(st)
    K = rng.uniform(0.0, 20.0, shape)
    sim.set_field(hca.FIELD_O2, K)
    K = sim.field(hca.FIELD_O2).astype(np.float64)       # as stored
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    u = rng.standard_normal(shape)
    u_stored = u.astype(sim.dtype).astype(np.float64)
    for which in range(4):
        got = sim.apply_operator(which, u).astype(np.float64)
        if which == 0:
            cpl, reac = S.o2_coupling(cfg), S.o2_reaction(st, K, cfg)
        else:
            cpl, reac = S.drug_coupling(cfg, which - 1), S.drug_reaction(st, perf, cfg, which - 1)
        ref = S.apply_operator(u_stored, cpl, reac)
        scale = operator_scale(cpl, reac, u_stored)
        err = np.max(np.abs(got - ref)) / scale
        assert err <= TOL[precision], (which, err)
    sim.close()


# rtol 1e-13 is near the attainable accuracy of FP64 CG on these operators, so
# iteration counts are compared at rtol 1e-10, where both runs stop on the
# same iteration unless rounding moves the crossing by one or two; values are
# compared at both tolerances (error <= cond(A) * rtol, cond(A) < 1e3 here).
RTOLS = [(1e-10, 1e-6, 3), (1e-13, 1e-9, None)]
# The drug operator's diagonal (~600/min) dwarfs its mass term 1/dt, so the
# rounding of x alone leaves a relative residual near 2e-12 in FP64: the tight
# drug solve stops at 1e-11 (error <= cond(A) * rtol, cond(A) ~ 4e3).
DRUG_RTOLS = [(1e-10, 1e-6, 3), (1e-11, 1e-7, None)]


@pytest.mark.parametrize("rtol,vtol,itol", RTOLS)
@pytest.mark.parametrize("shape", SHAPES[:3])
def test_o2_solve_fp64(shape, rtol, vtol, itol, rng):
    sim, cfg, _ = make_pair(shape, "f64", seed=4, n_drugs=0, rtol_o2=rtol, picard_maxit=1)
    st = random_states(shape, rng)
    st.reshape(-1)[0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, shape)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, K_prev)
    sim.stage(hca.STAGE_O2)
    got = sim.field(hca.FIELD_O2)
    ref, info = o2_solve(st, K_prev, cfg)
    s = sim.stats()
    assert s["o2_rel_residual"] <= 2 * rtol
    assert np.max(np.abs(got - ref)) <= vtol * np.max(np.abs(ref))
    if itol is not None:
        assert abs(s["o2_iterations"] - info.iterations) <= itol
    sim.close()


@pytest.mark.parametrize("rtol,vtol,itol", DRUG_RTOLS)
@pytest.mark.parametrize("shape", SHAPES[:3])
def test_drug_solves_fp64(shape, rtol, vtol, itol, rng):
    sim, cfg, _ = make_pair(shape, "f64", seed=5, n_drugs=2, rtol_drug=rtol, picard_maxit=1,
                            uptake_G=(0.0, 0.1, 0.0))
    st = random_states(shape, rng)
    sim.set_states(st)
    sim.set_step(3)
    G_old = [rng.random(shape) * 0.5, rng.random(shape) * 0.2]
    for d in range(2):
        sim.set_field(hca.FIELD_DRUG[d], G_old[d])
    sim.stage(hca.STAGE_DRUGS)
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    from oracle.model import plasma_levels
    G0 = plasma_levels(cfg, 4 * cfg.dt)
    s = sim.stats()
    for d in range(2):
        ref, info = drug_solve(st, perf, G_old[d], G0[d], cfg, d)
        got = sim.field(hca.FIELD_DRUG[d])
        assert s["drug_rel_residual"][d] <= 2 * rtol
        assert np.max(np.abs(got - ref)) <= vtol * max(1.0, np.max(np.abs(ref)))
        if itol is not None:
            assert abs(s["drug_iterations"][d] - info.iterations) <= itol
    sim.close()


def fp32_solve_case(shape, rng, **params):
    sim, cfg, _ = make_pair(shape, "f32", seed=6, n_drugs=1, picard_maxit=1, **params)
    st = random_states(shape, rng)
    st.reshape(-1)[0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, shape).astype(np.float32)
    G_old = (rng.random(shape) * 0.5).astype(np.float32)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, K_prev)
    sim.set_field(hca.FIELD_DRUG0, G_old)
    rc = sim.stage(hca.STAGE_O2 | hca.STAGE_DRUGS, allow_noconv=True)
    s = sim.stats()
    # the FP32 path's operator has FP32 coefficients; the oracle solves the
    # FP64 system to its attainable accuracy
    cfg64 = cfg.replace(precision="f64", rtol_o2=1e-13, rtol_drug=1e-11)
    refK, _ = o2_solve(st, K_prev.astype(np.float64), cfg64)
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    from oracle.model import plasma_levels
    refG, _ = drug_solve(st, perf, G_old.astype(np.float64), plasma_levels(cfg, cfg.dt)[0], cfg64, 0)
    errK = np.max(np.abs(sim.field(hca.FIELD_O2).astype(np.float64) - refK)) / np.max(np.abs(refK))
    errG = np.max(np.abs(sim.field(hca.FIELD_DRUG0).astype(np.float64) - refG)) / np.max(np.abs(refG))
    sim.close()
    return rc, s, errK, errG


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_fp32_defect_correction_reaches_fp64_tolerance(shape, rng):
    rc, s, errK, errG = fp32_solve_case(shape, rng, rtol_o2=1e-8, rtol_drug=1e-8, max_outer=10)
    print(f"defect correction: res K {s['o2_rel_residual']:.2e} G {s['drug_rel_residual'][0]:.2e}  "
          f"error vs FP64 oracle K {errK:.2e} G {errG:.2e}  sweeps {s['o2_sweeps']}")
    assert rc == hca.HCA_OK
    # the residual is measured to ~48 bits (float-float) on the two-word solution
    assert s["o2_rel_residual"] <= 1e-8 and s["drug_rel_residual"][0] <= 1e-8
    # fields agree with the FP64 oracle to the FP32 storage bar
    assert errK <= 1e-6 and errG <= 1e-6


@pytest.mark.parametrize("shape", SHAPES[1:3])
def test_fp32_defect_correction_decayed_field(shape, rng):
    # a drug washed out to ~1e-10 of its peak (epirubicin a day after a bolus):
    # the inner problem's residual is ~1e-22, so it must be rescaled to stay
    # clear of FP32 underflow
    sim, cfg, _ = make_pair(shape, "f32", seed=9, n_drugs=2, picard_maxit=1, rtol_drug=1e-8, max_outer=10)
    st = random_states(shape, rng)
    sim.set_states(st)
    sim.set_step(30)
    G_old = (rng.random(shape) * 1e-10).astype(np.float32)
    sim.set_field(hca.FIELD_DRUG1, G_old)
    rc = sim.stage(hca.STAGE_DRUGS)
    s = sim.stats()
    assert rc == hca.HCA_OK and s["drug_rel_residual"][1] <= 1e-8
    assert s["drug_iterations"][1] < 2000, s["drug_iterations"]
    from oracle.model import plasma_levels
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    cfg64 = cfg.replace(precision="f64", rtol_drug=1e-11)
    ref, _ = drug_solve(st, perf, G_old.astype(np.float64), plasma_levels(cfg, 31 * cfg.dt)[1], cfg64, 1)
    got = sim.field(hca.FIELD_DRUG1).astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))
    sim.close()


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_fp32_plain_cg_error(shape, rng):
    # plain FP32 CG (no defect correction): the stored-FP32 residual floor of
    # the drug operator is ~1e-3, so only the field error is asserted; the
    # drug solve stagnates at the FP32 floor, whose field error is of order
    # cond(D^-1 A) * eps_32 ~ 5e3 * 6e-8 = 3e-4, and the oxygen solve stops at
    # rtol 1e-6, whose field error is bounded by cond(A) * 1e-6 (both move
    # with the rounding of the CG passes)
    rc, s, errK, errG = fp32_solve_case(shape, rng, rtol_o2=1e-6, rtol_drug=1e-6, max_outer=0)
    print(f"plain fp32: res K {s['o2_rel_residual']:.2e} G {s['drug_rel_residual'][0]:.2e}  "
          f"error vs FP64 oracle K {errK:.2e} G {errG:.2e}")
    assert s["o2_rel_residual"] <= 2e-6
    assert errK <= 3e-4 and errG <= 3e-4


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES[:3])
def test_ode_update(shape, precision, rng):
    sim, cfg, _ = make_pair(shape, precision, seed=7, n_drugs=1, picard_maxit=1)
    st = random_states(shape, rng)
    K = rng.uniform(0.0, 20.0, shape)
    K.reshape(-1)[:5] = 0.0
    phi = rng.random(shape)
    P = rng.random(shape) * 0.1
    Vc = rng.random(shape) * 0.3
    sim.set_states(st)
    for bit, v in ((hca.FIELD_O2, K), (hca.FIELD_PHI, phi), (hca.FIELD_P53, P), (hca.FIELD_VEGFC, Vc)):
        sim.set_field(bit, v)
    stored = {b: sim.field(b).astype(np.float64) for b in (hca.FIELD_O2, hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC)}
    sim.stage(hca.STAGE_ODE)
    ref = ode_update(st, stored[hca.FIELD_PHI], stored[hca.FIELD_P53], stored[hca.FIELD_VEGFC],
                     stored[hca.FIELD_O2], cfg)
    for got_bit, r in zip((hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC), ref):
        got = sim.field(got_bit).astype(np.float64)
        rel = np.max(np.abs(got - r) / np.maximum(np.abs(r), 1e-3 * np.max(np.abs(r))))
        assert rel <= (1e-12 if precision == "f64" else 2e-6), (got_bit, rel)
    sim.close()


def ca_case(shape, precision, rng, threads=0, step=9, seed=21, n_drugs=2, kill_b=(1, 2, 1)):
    sim, cfg, _ = make_pair(shape, precision, threads=threads, seed=seed, n_drugs=n_drugs,
                            kill_b=kill_b, picard_maxit=1)
    st = random_states(shape, rng, p_vessel=0.05, p_cancer=0.55)
    phi = rng.random(shape) * 1.6
    K = rng.integers(0, 6, shape).astype(np.float64) + (rng.random(shape) < 0.5) * rng.random(shape)
    G = [rng.random(shape) * 0.6, rng.random(shape) * 0.4]
    P = rng.random(shape)
    Vc = rng.random(shape)
    return sim, cfg, st, phi, K, G[:n_drugs], P, Vc


def run_ca_both(sim, cfg, st, phi, K, G, P, Vc, step):
    sim.set_states(st)
    for bit, v in ((hca.FIELD_O2, K), (hca.FIELD_PHI, phi), (hca.FIELD_P53, P), (hca.FIELD_VEGFC, Vc)):
        sim.set_field(bit, v)
    for d, g in enumerate(G):
        sim.set_field(hca.FIELD_DRUG[d], g)
    stored = lambda b: sim.field(b).astype(np.float64)
    K_s, phi_s, P_s, V_s = (stored(b) for b in (hca.FIELD_O2, hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC))
    G_s = [stored(hca.FIELD_DRUG[d]) for d in range(len(G))]
    sim.set_step(step)
    sim.stage(hca.STAGE_CA)
    ref = ca_update(st, phi_s, P_s, V_s, K_s, G_s, cfg, step)
    return ref, sim.states(), stored(hca.FIELD_PHI), stored(hca.FIELD_P53), stored(hca.FIELD_VEGFC), sim.stats()


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_ca_bit_exact_given_fields(shape, precision, rng):
    for trial in range(3):
        sim, cfg, st, phi, K, G, P, Vc = ca_case(shape, precision, rng, seed=21 + trial)
        ref, gst, gphi, gP, gV, s = run_ca_both(sim, cfg, st, phi, K, G, P, Vc, step=9 + trial)
        assert np.array_equal(gst, ref[0])
        assert np.array_equal(gphi, ref[1].astype(sim.dtype).astype(np.float64))
        assert np.array_equal(gP, ref[2].astype(sim.dtype).astype(np.float64))
        assert np.array_equal(gV, ref[3].astype(sim.dtype).astype(np.float64))
        st_ref = ref[4]
        assert (s["committed"], s["kills"], s["divisions"], s["blocked"]) == (
            st_ref.committed, st_ref.kills, st_ref.divisions, st_ref.blocked)
        assert s["counts"] == np.bincount(ref[0].reshape(-1), minlength=6)[:6].tolist()
        sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_ca_tiling_invariance(precision):
    shape = (20, 33, 45)
    outs = []
    for threads in (64, 128, 256, 512):
        rng = np.random.default_rng(99)
        sim, cfg, st, phi, K, G, P, Vc = ca_case(shape, precision, rng, threads=threads)
        ref, gst, gphi, *_ = run_ca_both(sim, cfg, st, phi, K, G, P, Vc, step=4)
        outs.append((gst, gphi))
        sim.close()
    for gst, gphi in outs[1:]:
        assert np.array_equal(gst, outs[0][0]) and np.array_equal(gphi, outs[0][1])


def test_solver_bits_independent_of_block_size():
    shape = (24, 30, 42)
    results = []
    for threads in (64, 128, 256, 512):
        sim, cfg, _ = make_pair(shape, "f32", threads=threads, seed=8, n_drugs=2, rtol_o2=1e-6, rtol_drug=1e-6,
                                picard_tol=1e-5)
        sim.step(2)
        results.append([sim.field(b) for b in (hca.FIELD_O2, hca.FIELD_DRUG0, hca.FIELD_DRUG1, hca.FIELD_PHI)]
                       + [sim.states()])
        sim.close()
    for r in results[1:]:
        for a, b in zip(r, results[0]):
            assert np.array_equal(a, b)


def test_no_vessels_gives_zero_oxygen():
    shape = (6, 7, 9)
    sim, cfg, _ = make_pair(shape, "f64", seed=1, n_drugs=1, picard_maxit=1)
    st = np.full(shape, Pm.PROLIF, dtype=np.uint8)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, np.full(shape, 5.0))
    sim.stage(hca.STAGE_O2)
    assert np.all(sim.field(hca.FIELD_O2) == 0.0)
    assert sim.stats()["o2_rel_residual"] == 0.0
    sim.close()


def test_coupled_steps_fp64_match_oracle():
    n = 16
    params = dict(n_drugs=2, seed=12, rtol_o2=1e-13, rtol_drug=1e-13, picard_tol=1e-12)
    maps = make_maps(n, n, n, corr_len=3.0, seed=12)
    sim = hca.Sim.create(n, n, n, maps.p_cell, maps.perf, maps.p_vessel, **params)
    orc = OracleSim(Pm.Config(nx=n, ny=n, nz=n, **params), maps.p_cell, maps.perf, maps.p_vessel)
    assert np.max(np.abs(sim.field(hca.FIELD_O2) - orc.K)) <= 1e-9 * orc.K.max()
    for step in range(4):
        sim.step(1)
        orc.step(1)
        assert np.array_equal(sim.states(), orc.state), f"states differ after step {step}"
        for bit, ref in ((hca.FIELD_O2, orc.K), (hca.FIELD_DRUG0, orc.G[0]), (hca.FIELD_DRUG1, orc.G[1]),
                         (hca.FIELD_PHI, orc.phi), (hca.FIELD_P53, orc.P), (hca.FIELD_VEGFC, orc.Vc)):
            got = sim.field(bit)
            assert np.max(np.abs(got - ref)) <= 1e-9 * max(1e-3, np.max(np.abs(ref))), (step, bit)
        s = sim.stats()
        h = orc.history[-1]
        assert (s["kills"], s["divisions"], s["blocked"]) == (h.kills, h.divisions, h.blocked)
    sim.close()


def test_errors_are_reported():
    shape = (4, 4, 4)
    maps = make_maps(4, 4, 4, corr_len=1.0, seed=0)
    bad = maps.p_cell.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(hca.HcaError) as e:
        hca.Sim.create(4, 4, 4, bad, maps.perf, maps.p_vessel)
    assert e.value.status == hca.HCA_ERR_NONFINITE
    sim = hca.Sim.create(4, 4, 4, maps.p_cell, maps.perf, maps.p_vessel, n_drugs=1, maxit=1,
                         rtol_drug=1e-14, picard_maxit=1)
    sim.set_field(hca.FIELD_DRUG0, np.random.default_rng(0).random(shape))
    rc = sim.step(1, allow_noconv=True)
    assert rc == hca.HCA_ERR_NOCONV
    assert sim.stats()["not_converged"] & 2
    with pytest.raises(hca.HcaError):
        sim.field(hca.FIELD_DRUG1)            # drug 1 does not exist here
    short = np.empty(10, dtype=np.float64)
    with pytest.raises(hca.HcaError):
        hca.hca_read_fields(sim.handle, 0, hca.FIELD_O2, short)
    sim.close()


@pytest.mark.parametrize("pc", [0, 1])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_equals_single_replicates(precision, pc):
    # uneven lattices, distinct seeds and maps, one launch per kernel for all;
    # pc = 1: every replicate has its own multigrid hierarchy
    shapes = [(12, 16, 20), (8, 9, 13), (16, 16, 16)]
    params = dict(n_drugs=2, rtol_o2=1e-8, rtol_drug=1e-8, picard_tol=1e-7, preconditioner=pc)
    cfgs, maps = [], []
    for r, (nz, ny, nx) in enumerate(shapes):
        m = make_maps(nx, ny, nz, corr_len=3.0, seed=100 + r)
        maps.append((m.p_cell, m.perf, m.p_vessel))
        cfgs.append(hca.make_config(nx, ny, nz, precision=precision, seed=100 + r, **params))
    batch = hca.Sim(cfgs, maps, batch=True)
    batch.step(3)
    for r, (nz, ny, nx) in enumerate(shapes):
        single = hca.Sim(hca.make_config(nx, ny, nz, precision=precision, seed=100 + r, **params), maps[r])
        single.step(3)
        assert np.array_equal(batch.states(r), single.states())
        for bit in (hca.FIELD_O2, hca.FIELD_DRUG0, hca.FIELD_DRUG1, hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC):
            assert np.array_equal(batch.field(bit, r), single.field(bit)), (r, bit)
        sb, ss = batch.stats(r), single.stats()
        for key in ("o2_iterations", "drug_iterations", "kills", "divisions", "counts"):
            assert sb[key] == ss[key], (r, key)
        single.close()
    batch.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_autotuned_launch_shape_gives_identical_results(precision, monkeypatch):
    """threads_per_block = 0: the library times candidate launch shapes at
    creation; the steps must be bit-identical to a fixed 128-thread handle."""
    shape = (24, 40, 64)
    runs = []
    for threads, tune in ((0, "0"), (128, "1")):
        monkeypatch.setenv("HCA_NO_TUNE", tune)
        sim, _, _ = make_pair(shape, precision, seed=12, n_drugs=1, threads=threads)
        t, r = hca.hca_get_launch_config(sim.handle)
        assert t in (64, 128, 256, 512) and r in (64, 80, 96, 128)
        if threads:
            assert t == 128
        sim.step(2)
        runs.append((sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG0), sim.stats()))
        sim.close()
    (s0, K0, G0, st0), (s1, K1, G1, st1) = runs
    assert np.array_equal(s0, s1) and np.array_equal(K0, K1) and np.array_equal(G0, G1)
    assert st0["o2_iterations"] == st1["o2_iterations"] and st0["drug_iterations"] == st1["drug_iterations"]


def test_same_call_sequence_on_library_and_oracle():
    """The library and the oracle driven through the same call names
    (hca_* / oracle_*): states bit-exact, fields within 1e-9 (FP64)."""
    from oracle import api

    n = 12
    params = dict(n_drugs=2, seed=17, rtol_o2=1e-13, rtol_drug=1e-13, picard_tol=1e-12)
    m = make_maps(n, n, n, corr_len=3.0, seed=17)
    h = hca.hca_create(hca.make_config(n, n, n, **params), m.p_cell, m.perf, m.p_vessel)
    o = api.oracle_create(Pm.Config(n, n, n, **params), m.p_cell, m.perf, m.p_vessel)
    mask = hca.FIELD_O2 | hca.FIELD_DRUG0 | hca.FIELD_DRUG1 | hca.FIELD_PHI
    for _ in range(3):
        assert hca.hca_step(h, 1) == hca.HCA_OK
        api.oracle_step(o, 1)
        st = np.empty(n ** 3, dtype=np.uint8)
        hca.hca_read_states(h, 0, st)
        assert np.array_equal(st, api.oracle_read_states(o, 0))
        f = np.empty(4 * n ** 3)
        hca.hca_read_fields(h, 0, mask, f)
        ref = api.oracle_read_fields(o, 0, mask)
        assert np.max(np.abs(f - ref)) <= 1e-9 * np.max(np.abs(ref))
    hca.hca_destroy(h)
    api.oracle_destroy(o)
