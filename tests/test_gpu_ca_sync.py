"""The synchronous CA update (ca_mode = 1: decisions on the lattice before
the update, a contested site to the highest phi, then the lowest index;
Section 2.5 and Algorithm 2) on the GPU against the oracle
(oracle.ca_sync.ca_update_sync), bit-exact, and the 2-D lattice (nz = 1: the
5-point Laplacian and the 8-site Moore neighbourhood) in both CA modes."""

import numpy as np
import pytest

from gpu_helpers import make_pair, random_states
from oracle import params as Pm
from oracle.ca_sync import ca_update_sync
from oracle.model import OracleSim
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu

SHAPES = [(5, 7, 13), (11, 29, 37), (1, 48, 70), (3, 3, 1)]


def _case(shape, precision, rng, seed):
    sim, cfg, _ = make_pair(shape, precision, seed=seed, n_drugs=2, kill_b=(1, 2, 1), picard_maxit=1, ca_mode=1)
    st = random_states(shape, rng, p_vessel=0.05, p_cancer=0.6)
    # phi on a grid of eighths so that equal-phi contests occur
    phi = np.round(rng.random(shape) * 1.6 * 8) / 8
    K = rng.integers(0, 6, shape).astype(np.float64) + (rng.random(shape) < 0.5) * rng.random(shape)
    G = [rng.random(shape) * 0.6, rng.random(shape) * 0.4]
    return sim, cfg, st, phi, K, G, rng.random(shape), rng.random(shape)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_sync_ca_bit_exact_given_fields(shape, precision, rng):
    for trial in range(3):
        sim, cfg, st, phi, K, G, P, Vc = _case(shape, precision, rng, 51 + trial)
        sim.set_states(st)
        for bit, v in ((hca.FIELD_O2, K), (hca.FIELD_PHI, phi), (hca.FIELD_P53, P), (hca.FIELD_VEGFC, Vc)):
            sim.set_field(bit, v)
        for d, g in enumerate(G):
            sim.set_field(hca.FIELD_DRUG[d], g)
        stored = lambda b: sim.field(b).astype(np.float64)
        K_s, phi_s, P_s, V_s = (stored(b) for b in (hca.FIELD_O2, hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC))
        G_s = [stored(hca.FIELD_DRUG[d]) for d in range(2)]
        sim.set_step(7 + trial)
        sim.stage(hca.STAGE_CA)
        ref = ca_update_sync(st, phi_s, P_s, V_s, K_s, G_s, cfg, 7 + trial)
        assert np.array_equal(sim.states(), ref[0])
        assert np.array_equal(stored(hca.FIELD_PHI), ref[1].astype(sim.dtype).astype(np.float64))
        assert np.array_equal(stored(hca.FIELD_P53), ref[2].astype(sim.dtype).astype(np.float64))
        assert np.array_equal(stored(hca.FIELD_VEGFC), ref[3].astype(sim.dtype).astype(np.float64))
        s, r = sim.stats(), ref[4]
        assert (s["committed"], s["kills"], s["divisions"], s["blocked"]) == (r.committed, r.kills, r.divisions,
                                                                              r.blocked)
        if shape == SHAPES[1]:
            assert r.blocked > 0 and r.divisions > 0 and r.kills > 0
        sim.close()


@pytest.mark.parametrize("ca_mode", [0, 1])
@pytest.mark.parametrize("dims", [(16, 16, 16), (1, 40, 64)])
def test_coupled_steps_match_oracle(dims, ca_mode):
    nz, ny, nx = dims
    params = dict(n_drugs=2, seed=52, rtol_o2=1e-13, rtol_drug=1e-13, picard_tol=1e-12, ca_mode=ca_mode)
    maps = make_maps(nx, ny, nz, corr_len=3.0, seed=52)
    sim = hca.Sim.create(nx, ny, nz, maps.p_cell, maps.perf, maps.p_vessel, **params)
    orc = OracleSim(Pm.Config(nx=nx, ny=ny, nz=nz, **params), maps.p_cell, maps.perf, maps.p_vessel)
    for step in range(4):
        sim.step(1)
        orc.step(1)
        assert np.array_equal(sim.states(), orc.state), f"states differ after step {step}"
        for bit, ref in ((hca.FIELD_O2, orc.K), (hca.FIELD_DRUG0, orc.G[0]), (hca.FIELD_PHI, orc.phi)):
            got = sim.field(bit)
            assert np.max(np.abs(got - ref)) <= 1e-9 * max(1e-3, np.max(np.abs(ref))), (step, bit)
        s, h = sim.stats(), orc.history[-1]
        assert (s["kills"], s["divisions"], s["blocked"]) == (h.kills, h.divisions, h.blocked)
    sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_sync_graph_host_and_batch_agree_bitwise(precision, monkeypatch):
    out = []
    for no_graph in ("0", "1"):
        monkeypatch.setenv("HCA_NO_GRAPH", no_graph)
        sim, _, _ = make_pair((24, 40, 56), precision, seed=53, n_drugs=1, ca_mode=1)
        sim.step(3)
        out.append((sim.states(), sim.field(hca.FIELD_PHI)))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    monkeypatch.setenv("HCA_NO_GRAPH", "0")
    sizes, cfgs, maps, single = [12, 20], [], [], []
    for r, n in enumerate(sizes):
        m = make_maps(n, n, n, corr_len=3.0, seed=60 + r)
        maps.append((m.p_cell, m.perf, m.p_vessel))
        cfgs.append(hca.make_config(n, n, n, precision=precision, seed=60 + r, n_drugs=1, ca_mode=1))
        s = hca.Sim(cfgs[-1], maps[-1])
        s.step(3)
        single.append(s.states())
        s.close()
    b = hca.Sim(cfgs, maps, batch=True)
    b.step(3)
    for r in range(2):
        assert np.array_equal(b.states(r), single[r])
    b.close()


def test_ca_mode_errors():
    maps = make_maps(8, 8, 8, corr_len=1.0, seed=0)
    with pytest.raises(hca.HcaError) as e:
        hca.Sim.create(8, 8, 8, maps.p_cell, maps.perf, maps.p_vessel, ca_mode=2)
    assert e.value.status == hca.HCA_ERR_ARG
    cfgs = [hca.make_config(8, 8, 8, ca_mode=v) for v in (0, 1)]
    with pytest.raises(hca.HcaError) as e:
        hca.Sim(cfgs, [(maps.p_cell, maps.perf, maps.p_vessel)] * 2, batch=True)
    assert e.value.status == hca.HCA_ERR_ARG
