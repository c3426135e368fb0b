"""Parity at the workloads' full sizes.

* The 48^3 FP64 configuration (one drug, 24 hourly steps, seed 0) against the
  oracle step by step: states bit-exact every step, fields within 1e-9 at the
  end (both solvers run to 1e-13 here so that no CA decision can flip on the
  last bits of a field; at the workload's 1e-8 the runs are compared
  statistically in test_gpu_statistics.py).
* The 256^3 bench workload in the bench's launch configuration (FP32 fields,
  multigrid-PCG, defect correction, autotuned launch shape) on outputs the
  oracle computes one by one (seeding of sampled sites, the ODE update of
  sampled cells, every decision of the first colour of the CA sweep, whose
  sites see the lattice before the update; a site it kills may receive a
  daughter from a later colour) and on
  properties that hold at any size (global source-sink balances of the
  oxygen and drug solves, conservation of cells through the CA update).
"""

import numpy as np
import pytest

import bench
from oracle import params as Pm
from oracle import stencil as S
from oracle.ca import NEIGHBOUR_OFFSETS, colour_of, survival_probability
from oracle.model import OracleSim, plasma_levels
from oracle.odes import ode_update
from oracle.philox import site_uniform
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu


def test_48cubed_fp64_24_steps_match_oracle():
    n, steps = 48, 24
    params = dict(n_drugs=1, seed=0, rtol_o2=1e-13, rtol_drug=1e-13, picard_tol=1e-12)
    maps = make_maps(n, n, n, corr_len=4.0, seed=0)
    sim = hca.Sim.create(n, n, n, maps.p_cell, maps.perf, maps.p_vessel, **params)
    orc = OracleSim(Pm.Config(nx=n, ny=n, nz=n, **params), maps.p_cell, maps.perf, maps.p_vessel)
    for step in range(steps):
        sim.step(1)
        orc.step(1)
        assert np.array_equal(sim.states(), orc.state), f"states differ after step {step}"
    for bit, ref in ((hca.FIELD_O2, orc.K), (hca.FIELD_DRUG0, orc.G[0]), (hca.FIELD_PHI, orc.phi),
                     (hca.FIELD_P53, orc.P), (hca.FIELD_VEGFC, orc.Vc)):
        got = sim.field(bit)
        assert np.max(np.abs(got - ref)) <= 1e-9 * max(1e-3, np.max(np.abs(ref))), bit
    sim.close()


@pytest.fixture(scope="module")
def bench_sim():
    n = bench.N_EDGE
    maps = make_maps(n, n, n, corr_len=bench.CORR_LEN, seed=bench.WORKLOAD["seed"])
    cfg = hca.make_config(n, n, n, **bench.WORKLOAD)
    sim = hca.Sim(cfg, (maps.p_cell, maps.perf, maps.p_vessel))
    ocfg = Pm.Config(nx=n, ny=n, nz=n, **{k: v for k, v in bench.WORKLOAD.items()
                                            if k in Pm.Config.__dataclass_fields__})
    yield sim, ocfg, maps
    sim.close()


def test_256cubed_seeding_of_sampled_sites(bench_sim):
    sim, cfg, maps = bench_sim
    rng = np.random.default_rng(0)
    sites = np.sort(rng.choice(cfg.n_sites, 20000, replace=False)).astype(np.uint64)
    u_v = site_uniform(cfg.seed, sites, 0, Pm.PURPOSE_VESSEL)
    u_c = site_uniform(cfg.seed, sites, 0, Pm.PURPOSE_CANCER)
    u_p = site_uniform(cfg.seed, sites, 0, Pm.PURPOSE_PHI)
    pv = maps.p_vessel.reshape(-1)[sites].astype(np.float64)
    pc = maps.p_cell.reshape(-1)[sites].astype(np.float64)
    want = np.where(u_v < pv, Pm.VESSEL, np.where(u_c < pc, Pm.PROLIF, Pm.EMPTY))
    assert np.array_equal(sim.states().reshape(-1)[sites], want)
    phi = sim.field(hca.FIELD_PHI).reshape(-1)[sites]
    assert np.array_equal(phi, np.where(want == Pm.PROLIF, u_p, 0.0).astype(np.float32))


def test_256cubed_one_step_by_stages(bench_sim):
    sim, cfg, _ = bench_sim
    sim.step(2)                                  # leave the seeded state
    st = sim.states()
    perf = sim.field(hca.FIELD_PERF).astype(np.float64)
    # oxygen: sum_i a_i(K_prev) K_i = sum_i b_i (the Laplacian's rows sum to zero
    # under Neumann boundaries), independent of the FP32 rounding of K
    K_prev = sim.field(hca.FIELD_O2).astype(np.float64)
    sim.stage(hca.STAGE_O2)
    K = sim.field(hca.FIELD_O2).astype(np.float64)
    a = S.o2_reaction(st, K_prev, cfg)
    b = S.o2_rhs(st, cfg)
    assert abs(np.sum(a * K) - np.sum(b)) <= 1e-6 * np.sum(b)
    # discrete maximum principle (to the solver tolerance)
    assert K.min() >= -1e-6 * cfg.K0 and K.max() <= cfg.K0 * (1 + 1e-6)
    # drugs: the same balance for each implicit-Euler step
    step = sim.stats()["step"]
    G_old = [sim.field(hca.FIELD_DRUG[d]).astype(np.float64) for d in range(cfg.n_drugs)]
    sim.stage(hca.STAGE_DRUGS)
    for d, G0 in enumerate(plasma_levels(cfg, (step + 1) * cfg.dt)):
        G = sim.field(hca.FIELD_DRUG[d]).astype(np.float64)
        a = S.drug_reaction(st, perf, cfg, d)
        b = S.drug_rhs(st, perf, G_old[d], G0, cfg, d)
        assert abs(np.sum(a * G) - np.sum(b)) <= 1e-6 * abs(np.sum(b)), d
    # ODEs on sampled cells, one by one
    phi0, P0, V0 = (sim.field(b).astype(np.float64) for b in (hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC))
    sim.stage(hca.STAGE_ODE)
    cells = np.flatnonzero(np.isin(st.reshape(-1), Pm.CONSUMER_STATES))
    pick = np.random.default_rng(1).choice(cells, 5000, replace=False)
    ref = ode_update(st.reshape(-1)[pick], phi0.reshape(-1)[pick], P0.reshape(-1)[pick], V0.reshape(-1)[pick],
                     K.astype(np.float32).astype(np.float64).reshape(-1)[pick], cfg)
    for bit, r in zip((hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC), ref):
        got = sim.field(bit).astype(np.float64).reshape(-1)[pick]
        assert np.max(np.abs(got - r) / np.maximum(np.abs(r), 1e-3)) <= 2e-6, bit
    # CA: every decision of colour 0 (which sees the lattice before the update)
    # recomputed one by one, and cell conservation over the whole sweep
    st0 = st.reshape(-1).copy()
    st0[st0 == Pm.DEAD] = Pm.EMPTY
    phi1 = sim.field(hca.FIELD_PHI).reshape(-1)
    Kf = sim.field(hca.FIELD_O2).reshape(-1)
    Gf = [sim.field(hca.FIELD_DRUG[d]).reshape(-1) for d in range(cfg.n_drugs)]
    nz, ny, nx = st.shape
    sim.stage(hca.STAGE_CA)
    after = sim.states().reshape(-1)
    s = sim.stats()
    live = lambda v: int(np.isin(v, Pm.CANCER_STATES).sum())
    assert live(after) == live(st0) - s["kills"] + s["divisions"]
    committed = np.flatnonzero(np.isin(st0, Pm.CANCER_STATES) & (phi1 >= np.float32(1)))
    z, rem = np.divmod(committed, nx * ny)
    y, x = np.divmod(rem, nx)
    first = committed[colour_of(x, y, z) == 0]
    assert first.size > 100
    u = site_uniform(cfg.seed, first.astype(np.uint64), step, Pm.PURPOSE_KILL).astype(np.float32)
    kills0 = dead0 = 0
    for site, uk in zip(first.tolist(), u.tolist()):
        zz, r2 = divmod(site, nx * ny)
        yy, xx = divmod(r2, nx)
        p_kill = np.float32(np.float32(1) - survival_probability([g[site] for g in Gf], cfg, np.float32))
        if np.float32(uk) < p_kill:
            # killed: DEAD, unless a parent of a later colour placed a daughter on the freed site
            assert after[site] in (Pm.DEAD, Pm.PROLIF)
            kills0 += 1
            dead0 += int(after[site] == Pm.DEAD)
            continue
        best, bk = -1, None
        for dz, dy, dx in NEIGHBOUR_OFFSETS:
            a_, b_, c_ = xx + dx, yy + dy, zz + dz
            if 0 <= a_ < nx and 0 <= b_ < ny and 0 <= c_ < nz:
                nb = a_ + nx * (b_ + ny * c_)
                if st0[nb] in Pm.FREE_STATES and (best < 0 or Kf[nb] > bk):
                    best, bk = nb, Kf[nb]
        # a surviving parent is not committed again in this update, and a
        # daughter (phi = 0) is not either: their states are final
        if best >= 0:
            assert after[site] == Pm.PROLIF and after[best] == Pm.PROLIF
        else:
            assert after[site] == Pm.QUIESC
    if kills0:
        assert dead0 >= 0.5 * kills0
