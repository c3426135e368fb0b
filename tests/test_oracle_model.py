"""Pins for the oracle's initialisation and a short coupled run, plus the map recipe."""

import math

import numpy as np

from oracle import params as Pm
from oracle.model import OracleSim, plasma_levels, seed_lattice
from synth import make_maps, replicate_sizes


def test_seeding_binomial():
    n = 40
    cfg = Pm.Config(nx=n, ny=n, nz=n, seed=4)
    pc = np.full(cfg.shape, 0.4, dtype=np.float32)
    pv = np.full(cfg.shape, 0.12, dtype=np.float32)
    state, phi = seed_lattice(cfg, pc, pv)
    N = n ** 3
    nv = (state == Pm.VESSEL).sum()
    assert abs(nv - 0.12 * N) < 4 * math.sqrt(N * 0.12 * 0.88)
    free = N - nv
    nc = (state == Pm.PROLIF).sum()
    assert abs(nc - 0.4 * free) < 4 * math.sqrt(free * 0.4 * 0.6)
    # phi ~ U(0, 1) on cancer cells only
    ph = phi[state == Pm.PROLIF]
    assert np.all((ph >= 0) & (ph < 1))
    assert abs(ph.mean() - 0.5) < 4 * math.sqrt(1 / 12 / ph.size)
    assert np.all(phi[state != Pm.PROLIF] == 0)


def test_seeding_follows_maps():
    n = 32
    cfg = Pm.Config(nx=n, ny=n, nz=n, seed=5)
    pc = np.zeros(cfg.shape, dtype=np.float32)
    pc[:, :, : n // 2] = 1.0
    pv = np.zeros(cfg.shape, dtype=np.float32)
    state, _ = seed_lattice(cfg, pc, pv)
    assert np.all(state[:, :, : n // 2] == Pm.PROLIF)
    assert np.all(state[:, :, n // 2:] == Pm.EMPTY)


def test_short_coupled_run_invariants():
    n = 12
    cfg = Pm.Config(nx=n, ny=n, nz=n, n_drugs=2, seed=0, rtol_o2=1e-10, rtol_drug=1e-10)
    maps = make_maps(n, n, n, corr_len=3.0, seed=0)
    sim = OracleSim(cfg, maps.p_cell, maps.perf, maps.p_vessel)
    assert 0.0 <= sim.K.min() and sim.K.max() <= cfg.K0
    cells0 = np.isin(sim.state, Pm.CANCER_STATES).sum()
    total_div = total_kill = 0
    for _ in range(3):
        st = sim.step()
        assert st.o2.converged and all(d.converged for d in st.drugs)
        assert st.o2.rel_residual < 1e-9
        total_div += st.divisions
        total_kill += st.kills
        assert st.counts.sum() == n ** 3
    cells = np.isin(sim.state, Pm.CANCER_STATES).sum()
    assert cells - cells0 == total_div - total_kill
    assert np.all(sim.G[0] >= -1e-12) and np.all(sim.G[0] <= 1.0 + 1e-12)
    # vessels are static on this path
    st0, _ = seed_lattice(cfg, maps.p_cell, maps.p_vessel)
    assert np.array_equal(sim.state == Pm.VESSEL, st0 == Pm.VESSEL)


def test_plasma_levels_schedule():
    cfg = Pm.Config(nx=1, ny=1, nz=1, n_drugs=2, dose_interval=21, dt=60.0)
    g = plasma_levels(cfg, 60.0)
    assert math.isclose(g[0], math.exp(-cfg.plasma_decay[0] * 60.0))
    g21 = plasma_levels(cfg, 21 * 60.0)
    assert math.isclose(g21[1], 1.0 + math.exp(-cfg.plasma_decay[1] * 21 * 60.0))


def test_map_recipe_statistics():
    m = make_maps(64, 64, 64, corr_len=4.0, seed=1)
    assert m.p_cell.dtype == np.float32 and m.p_cell.shape == (64, 64, 64)
    assert abs(m.p_cell.mean() - 0.4) < 0.02
    assert abs(m.perf.mean() - 1.0) < 0.05
    assert abs(m.p_vessel.mean() - 0.12) < 0.01
    assert m.p_cell.min() >= 0 and m.p_cell.max() <= 1
    # smoothing: neighbouring sites are strongly correlated, distant ones are not
    a = m.p_cell
    near = np.corrcoef(a[:, :, :-1].ravel(), a[:, :, 1:].ravel())[0, 1]
    far = np.corrcoef(a[:, :, :-32].ravel(), a[:, :, 32:].ravel())[0, 1]
    assert near > 0.9 and abs(far) < 0.1
    again = make_maps(64, 64, 64, corr_len=4.0, seed=1)
    assert np.array_equal(again.perf, m.perf)


def test_replicate_sizes():
    s = replicate_sizes(64)
    assert len(s) == 64 and set(s) <= {64, 96, 128, 192}
    assert s == replicate_sizes(64)
