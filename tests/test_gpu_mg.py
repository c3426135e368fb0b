"""GPU parity of the multigrid-preconditioned CG (HCA_PC_MG) with the FP64
oracle in oracle/multigrid.py: the V-cycle z = M r on the operators of both
equations, MG-PCG solves (iteration counts and fields), FP32 with defect
correction, the graph and host-loop paths, and edge cases.

Tolerance of z = M r (FP64): 1e-10 relative.  The GPU recovers the
reaction coefficient on level 0 as d - c n from the stored diagonal; for the
drug operator d ~ 576 and a ~ 0.027, so that subtraction carries ~1e-13
absolute (4e-12 relative) error into the coarse diagonals; every other
difference is summation order.
"""

import os

import numpy as np
import pytest

from gpu_helpers import make_pair, random_states
from oracle import multigrid as MG
from oracle import params as Pm
from oracle import stencil as S
from oracle.model import plasma_levels
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu

# (nz, ny, nx): one level (<= 512 sites), two and three levels with the
# coarse part in the single-block kernel, four levels with a grid-kernel level,
# a flat lattice (in-plane coarsening), one that becomes flat after a level,
# and odd extents on every axis (a last fine row or plane alone in its
# coarse cell) with two and three levels
SHAPES = [(5, 7, 13), (16, 16, 16), (32, 32, 32), (24, 40, 56), (1, 48, 70), (2, 40, 60), (9, 13, 21),
          (17, 23, 31)]


def _operator(which, st, K, perf, cfg):
    if which == 0:
        return S.o2_coupling(cfg), S.o2_reaction(st, K, cfg)
    return S.drug_coupling(cfg, which - 1), S.drug_reaction(st, perf, cfg, which - 1)


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_vcycle_matches_oracle(shape, which, rng):
    sim, cfg, _ = make_pair(shape, "f64", seed=2, n_drugs=1, preconditioner=hca.HCA_PC_MG, picard_maxit=1)
    st = random_states(shape, rng)
    K = rng.uniform(0.0, 20.0, shape)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, K)
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    r = rng.standard_normal(shape)
    z = sim.apply_preconditioner(which, r)
    sim.close()
    c, a = _operator(which, st, K, perf, cfg)
    ref = MG.vcycle(MG.hierarchy(c, a), r)
    assert np.max(np.abs(z - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", SHAPES[1:])
def test_mg_pcg_oxygen_matches_oracle(shape, rng):
    rtol = 1e-10
    sim, cfg, _ = make_pair(shape, "f64", seed=4, n_drugs=0, rtol_o2=rtol, picard_maxit=1,
                            preconditioner=hca.HCA_PC_MG)
    st = random_states(shape, rng)
    st.reshape(-1)[0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, shape)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, K_prev)
    sim.stage(hca.STAGE_O2)
    got = sim.field(hca.FIELD_O2)
    s = sim.stats()
    sim.close()
    c, a = _operator(0, st, K_prev, None, cfg)
    ref, info = MG.mg_pcg(c, a, S.o2_rhs(st, cfg), K_prev, rtol, 1000)
    assert s["o2_rel_residual"] <= 2 * rtol
    assert abs(s["o2_iterations"] - info.iterations) <= 1
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", SHAPES[1:])
def test_mg_pcg_drug_matches_oracle(shape, rng):
    rtol = 1e-10
    sim, cfg, _ = make_pair(shape, "f64", seed=5, n_drugs=1, rtol_drug=rtol, picard_maxit=1,
                            preconditioner=hca.HCA_PC_MG)
    st = random_states(shape, rng)
    sim.set_states(st)
    sim.set_step(3)
    G_old = rng.random(shape) * 0.5
    sim.set_field(hca.FIELD_DRUG[0], G_old)
    sim.stage(hca.STAGE_DRUGS)
    got = sim.field(hca.FIELD_DRUG[0])
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    s = sim.stats()
    sim.close()
    G0 = plasma_levels(cfg, 4 * cfg.dt)[0]
    c, a = _operator(1, st, None, perf, cfg)
    ref, info = MG.mg_pcg(c, a, S.drug_rhs(st, perf, G_old, G0, cfg, 0), G_old, rtol, 1000)
    assert s["drug_rel_residual"][0] <= 2 * rtol
    assert abs(s["drug_iterations"][0] - info.iterations) <= 1
    assert np.max(np.abs(got - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))


def test_mg_cuts_drug_iterations(rng):
    shape = (32, 32, 32)
    its = {}
    for pc in (hca.HCA_PC_JACOBI, hca.HCA_PC_MG):
        sim, cfg, _ = make_pair(shape, "f64", seed=5, n_drugs=1, rtol_drug=1e-8, picard_maxit=1, preconditioner=pc)
        sim.set_step(3)
        sim.set_field(hca.FIELD_DRUG[0], np.zeros(shape))
        sim.stage(hca.STAGE_DRUGS)
        its[pc] = sim.stats()["drug_iterations"][0]
        sim.close()
    assert its[hca.HCA_PC_MG] * 5 < its[hca.HCA_PC_JACOBI]


@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 40, 56)])
def test_fp32_defect_correction_with_mg(shape, rng):
    """FP32 storage, FP32 inner MG-PCG, float-float residuals: the field matches the
    FP64 oracle within the FP32 bound (1e-6 relative)."""
    sim, cfg, _ = make_pair(shape, "f32", seed=6, n_drugs=1, rtol_o2=1e-8, rtol_drug=1e-8, picard_maxit=1,
                            preconditioner=hca.HCA_PC_MG)
    st = random_states(shape, rng)
    st.reshape(-1)[0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, shape).astype(np.float32)
    G_old = (rng.random(shape) * 0.5).astype(np.float32)
    sim.set_states(st)
    sim.set_step(3)
    sim.set_field(hca.FIELD_O2, K_prev)
    sim.set_field(hca.FIELD_DRUG[0], G_old)
    sim.stage(hca.STAGE_O2 | hca.STAGE_DRUGS)
    K, G = sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG[0])
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    s = sim.stats()
    sim.close()
    cK, aK = _operator(0, st, K_prev.astype(np.float64), None, cfg)
    refK, _ = MG.mg_pcg(cK, aK, S.o2_rhs(st, cfg), K_prev.astype(np.float64), 1e-12, 1000)
    G0 = plasma_levels(cfg, 4 * cfg.dt)[0]
    cG, aG = _operator(1, st, None, perf, cfg)
    refG, _ = MG.mg_pcg(cG, aG, S.drug_rhs(st, perf, G_old.astype(np.float64), G0, cfg, 0),
                        G_old.astype(np.float64), 1e-12, 1000)
    assert s["o2_rel_residual"] <= 1e-8 and s["drug_rel_residual"][0] <= 1e-8
    assert np.max(np.abs(K - refK)) <= 1e-6 * np.max(np.abs(refK))
    assert np.max(np.abs(G - refG)) <= 1e-6 * max(1.0, np.max(np.abs(refG)))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_graph_and_host_loop_agree_bitwise(precision, monkeypatch):
    shape = (24, 40, 56)
    out = []
    for no_graph in ("0", "1"):
        monkeypatch.setenv("HCA_NO_GRAPH", no_graph)
        sim, _, _ = make_pair(shape, precision, seed=8, n_drugs=2, preconditioner=hca.HCA_PC_MG)
        sim.step(3)
        out.append((sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG[0]), sim.stats()))
        sim.close()
    (s0, K0, G0, st0), (s1, K1, G1, st1) = out
    assert np.array_equal(s0, s1) and np.array_equal(K0, K1) and np.array_equal(G0, G1)
    assert st0["o2_iterations"] == st1["o2_iterations"]
    assert st0["drug_iterations"] == st1["drug_iterations"]


def test_coupled_steps_match_jacobi(rng):
    """Same coupled run with both preconditioners (FP64, 1e-10): the fields
    agree to the solver tolerance and the CA takes the same decisions."""
    shape = (24, 32, 40)
    res = []
    for pc in (hca.HCA_PC_JACOBI, hca.HCA_PC_MG):
        sim, _, _ = make_pair(shape, "f64", seed=9, n_drugs=1, rtol_o2=1e-10, rtol_drug=1e-10, preconditioner=pc)
        sim.step(4)
        res.append((sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG[0])))
        sim.close()
    (sa, Ka, Ga), (sb, Kb, Gb) = res
    assert np.max(np.abs(Ka - Kb)) <= 1e-8 * np.max(np.abs(Ka))
    assert np.max(np.abs(Ga - Gb)) <= 1e-8 * max(1.0, np.max(np.abs(Ga)))
    assert np.mean(sa != sb) <= 1e-4


def test_mg_edge_cases():
    # no vessels: b = 0, K = 0 exactly
    sim, _, _ = make_pair((16, 16, 16), "f64", seed=1, n_drugs=0, preconditioner=hca.HCA_PC_MG, picard_maxit=1)
    st = np.full((16, 16, 16), Pm.PROLIF, dtype=np.uint8)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, np.full((16, 16, 16), 7.0))
    sim.stage(hca.STAGE_O2)
    assert np.all(sim.field(hca.FIELD_O2) == 0.0)
    sim.close()
    # a lattice of at most 512 sites is its own coarsest level
    sim, cfg, _ = make_pair((1, 20, 25), "f64", seed=1, n_drugs=0, rtol_o2=1e-10, preconditioner=hca.HCA_PC_MG)
    sim.step(1)
    assert sim.stats()["o2_rel_residual"] <= 2e-10
    sim.close()
    # a batch needs a coarse level in every replicate (a 6x6x6 lattice has none)
    cfgs, maps = [], []
    for n in (16, 6):
        m = [np.full((n, n, n), 0.5, dtype=np.float32)] * 3
        maps.append(m)
        cfgs.append(hca.make_config(n, n, n, preconditioner=hca.HCA_PC_MG))
    with pytest.raises(hca.HcaError) as e:
        hca.Sim(cfgs, maps, batch=True)
    assert e.value.status == hca.HCA_ERR_UNIMPLEMENTED
    # an invalid preconditioner and the Jacobi-only entry point
    with pytest.raises(hca.HcaError) as e:
        sim = hca.Sim.create(8, 8, 8, *[np.full((8, 8, 8), 0.5, dtype=np.float32)] * 3, preconditioner=7)
    assert e.value.status == hca.HCA_ERR_ARG
    sim, _, _ = make_pair((8, 8, 8), "f64", seed=1, n_drugs=0)
    with pytest.raises(hca.HcaError) as e:
        sim.apply_preconditioner(0, np.zeros((8, 8, 8)))
    assert e.value.status == hca.HCA_ERR_STATE
    sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 40, 56), (20, 44, 104), (1, 64, 96)])
def test_row_coarse_kernels_are_bit_identical(shape, precision, monkeypatch):
    """The row-vector coarse post-sweep gives the per-site kernel's bits."""
    out = []
    for generic in ("1", "0"):
        monkeypatch.setenv("HCA_MG_GENERIC", generic)
        sim, _, _ = make_pair(shape, precision, seed=13, n_drugs=2, preconditioner=hca.HCA_PC_MG)
        sim.step(2)
        out.append((sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG[1]), sim.stats()))
        sim.close()
    (s0, K0, G0, st0), (s1, K1, G1, st1) = out
    assert np.array_equal(s0, s1) and np.array_equal(K0, K1) and np.array_equal(G0, G1)
    assert (st0["o2_iterations"], st0["drug_iterations"]) == (st1["o2_iterations"], st1["drug_iterations"])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_row_coarse_kernels_batch_bit_identical(precision, monkeypatch):
    """Batches (replicates of several sizes, item prefix tables per level)
    give the per-site coarse kernels' bits too."""
    res = []
    for generic in ("1", "0"):
        monkeypatch.setenv("HCA_MG_GENERIC", generic)
        cfgs, maps = [], []
        for r, n in enumerate((48, 40, 64)):
            m = make_maps(n, n, n, corr_len=3.0, seed=80 + r)
            maps.append((m.p_cell, m.perf, m.p_vessel))
            cfgs.append(hca.make_config(n, n, n, precision=precision, seed=80 + r, n_drugs=1,
                                        preconditioner=hca.HCA_PC_MG))
        b = hca.Sim(cfgs, maps, batch=True)
        b.step(2)
        res.append([(b.states(r), b.field(hca.FIELD_O2, r), b.field(hca.FIELD_DRUG0, r)) for r in range(3)])
        b.close()
    for x, y in zip(*res):
        for a, c in zip(x, y):
            assert np.array_equal(a, c)
