"""The oracle's VEGF field (oracle.model.vegf_step), vascular automaton
(oracle.vascular) and pharmacokinetic models (oracle.pk) pinned by closed
forms, ODE integration, conservation and brute force."""

import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import model as M
from oracle import params as Pm
from oracle import pk
from oracle import stencil as S
from oracle.philox import site_uniform
from oracle.vascular import FIX, vascular_update


# ------------------------------------------------------------------ PK ---
@pytest.mark.parametrize("peak", [1.0, 54.0, 300.0])
def test_michaelis_menten_matches_ode_integration(peak):
    cfg = Pm.Config(4, 4, 4, pk_model=(0, 0, 1), dose_peak=(1.0, 1.0, peak), dose_interval=3, dt=60.0)
    rhs = lambda t, g: [-cfg.mm_vmax * g[0] / (cfg.mm_km + g[0])]
    g, t0, ts = peak, 0.0, []
    for n in range(3):          # three doses, 180 min apart
        sol = solve_ivp(rhs, (t0, t0 + 180.0), [g], rtol=1e-12, atol=1e-14, dense_output=True)
        for t in (t0 + 1.0, t0 + 37.5, t0 + 179.0):
            ts.append((t, float(sol.sol(t)[0])))
        g = float(sol.y[0, -1]) + peak
        t0 += 180.0
    for t, ref in ts:
        assert abs(pk.plasma_level(cfg, 2, t) - ref) <= 1e-9 * peak


def test_michaelis_menten_linear_limit():
    """For G << k_m the model is the exponential with rate v_max / k_m."""
    cfg = Pm.Config(4, 4, 4, pk_model=(0, 0, 1), dose_peak=(1.0, 1.0, 1e-6))
    for t in (10.0, 100.0, 1000.0):
        ref = 1e-6 * math.exp(-cfg.mm_vmax / cfg.mm_km * t)
        assert abs(pk.plasma_level(cfg, 2, t) - ref) <= 1e-6 * ref


def test_three_compartment_matches_ode_and_conserves():
    cfg = Pm.Config(4, 4, 4, pk_model=(0, 2, 0), dose_interval=5, dt=60.0)
    Mx = pk.three_compartment_matrix(cfg)
    assert np.allclose(Mx.sum(axis=0), [-cfg.epi_cl2 / cfg.epi_w[0], 0.0, 0.0])   # loss only by elimination
    sol = solve_ivp(lambda t, a: Mx @ a, (0, 299.0), [1.0, 0.0, 0.0], rtol=1e-12, atol=1e-15, dense_output=True)
    for t in (0.5, 10.0, 123.0, 299.0):
        assert abs(pk.plasma_level(cfg, 1, t) - sol.sol(t)[0]) <= 1e-9
    # a second dose at t = 300 superposes
    t = 350.0
    ref = solve_ivp(lambda t, a: Mx @ a, (0, 350.0), [1.0, 0, 0], rtol=1e-12, atol=1e-15).y[0, -1] + \
        solve_ivp(lambda t, a: Mx @ a, (0, 50.0), [1.0, 0, 0], rtol=1e-12, atol=1e-15).y[0, -1]
    assert abs(pk.plasma_level(cfg, 1, t) - ref) <= 1e-8


# ---------------------------------------------------------------- VEGF ---
def test_vegf_uniform_source_closed_form():
    """All sites cells with equal Vc: V stays uniform and follows
    V^k = (V^{k-1}/h + a Vc) / (1/h + psi) per implicit-Euler sub-step."""
    shape = (4, 5, 6)
    cfg = Pm.Config(6, 5, 4, vegf=1, drug_substeps=3, rtol_drug=1e-14)
    st = np.full(shape, Pm.PROLIF, dtype=np.uint8)
    Vc = np.full(shape, 0.37)
    V = np.full(shape, 2e-5)
    got, infos = M.vegf_step(st, V, Vc, cfg)
    h = cfg.dt / 3
    v = 2e-5
    for _ in range(3):
        v = (v / h + cfg.a_V * 0.37) / (1 / h + cfg.psi_V)
    assert len(infos) == 3
    assert np.max(np.abs(got - v)) <= 1e-12 * v


def test_vegf_mass_balance():
    """Neumann boundaries: the total of V changes only by release and decay:
    sum V^k (1/h + psi) = sum V^{k-1}/h + a sum_cells Vc (implicit Euler)."""
    rng = np.random.default_rng(3)
    shape = (5, 6, 7)
    cfg = Pm.Config(7, 6, 5, vegf=1, rtol_drug=1e-14)
    st = rng.integers(0, 6, size=shape).astype(np.uint8)
    Vc = rng.random(shape)
    V0 = rng.random(shape) * 1e-4
    V, _ = M.vegf_step(st, V0, Vc, cfg)
    h = cfg.dt
    lhs = V.sum() * (1 / h + cfg.psi_V)
    rhs = V0.sum() / h + cfg.a_V * Vc[S.is_consumer(st)].sum()
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


# ------------------------------------------------------------ vessels ---
def _brute_vascular(state, V, cfg, step):
    """Site-by-site restatement with Python integers and floats."""
    st = state.reshape(-1).tolist()
    Vl = [float(v) for v in np.asarray(V, dtype=np.float64).reshape(-1)]
    n = len(st)
    s1 = sum(math.floor(v / (cfg.V_sprout + v) * FIX) for i, v in enumerate(Vl) if st[i] == Pm.VESSEL)
    ok = [cfg.V_low <= v <= cfg.V_high for v in Vl]
    s2 = sum(math.floor(Vl[i] / cfg.V_high * FIX) for i in range(n) if st[i] in (Pm.EMPTY, Pm.DEAD) and ok[i])
    u = site_uniform(cfg.seed, np.arange(n, dtype=np.uint64), step, Pm.PURPOSE_VASCULAR)
    out = list(st)
    for i in range(n):
        if st[i] == Pm.VESSEL and not ok[i] and u[i] < cfg.p_death:
            out[i] = Pm.EMPTY
        elif st[i] in (Pm.EMPTY, Pm.DEAD) and ok[i] and s2 > 0:
            if u[i] < min(1.0, cfg.beta_birth * float(s1) * (Vl[i] / cfg.V_high) / float(s2)):
                out[i] = Pm.VESSEL
    return np.array(out, dtype=np.uint8).reshape(state.shape)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vascular_update_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    shape = (6, 7, 8)
    cfg = Pm.Config(8, 7, 6, seed=seed, p_death=0.4, beta_birth=2.0)
    st = rng.choice([Pm.EMPTY, Pm.PROLIF, Pm.DEAD, Pm.VESSEL, Pm.STROMA], size=shape,
                    p=[0.4, 0.3, 0.05, 0.15, 0.1]).astype(np.uint8)
    V = 10 ** rng.uniform(-7, -2.5, shape)
    got, stats = vascular_update(st, V, cfg, 35)
    assert np.array_equal(got, _brute_vascular(st, V, cfg, 35))
    assert stats.births == int(((got == Pm.VESSEL) & (st != Pm.VESSEL)).sum())
    assert stats.deaths == int(((got != Pm.VESSEL) & (st == Pm.VESSEL)).sum())
    assert stats.births > 0 and stats.deaths > 0


def test_vascular_probabilities():
    """p_death = 1 removes every out-of-range vessel and none in range;
    the expected number of births equals E[n_new] when no p is clipped."""
    shape = (10, 20, 30)
    rng = np.random.default_rng(5)
    st = np.where(rng.random(shape) < 0.1, Pm.VESSEL, Pm.EMPTY).astype(np.uint8)
    V = 10 ** rng.uniform(-7, -2.5, shape)
    cfg = Pm.Config(30, 20, 10, p_death=1.0, beta_birth=0.02)
    got, stats = vascular_update(st, V, cfg, 3)
    inr = (V >= cfg.V_low) & (V <= cfg.V_high)
    assert np.all(got[(st == Pm.VESSEL) & ~inr] == Pm.EMPTY)
    assert np.all(got[(st == Pm.VESSEL) & inr] == Pm.VESSEL)
    ves = st == Pm.VESSEL
    expected = cfg.beta_birth * np.sum(V[ves] / (cfg.V_sprout + V[ves]))
    births = []
    for step in range(200):
        births.append(vascular_update(st, V, cfg, step)[1].births)
    mean = np.mean(births)
    assert abs(mean - expected) <= 4 * math.sqrt(expected / 200) + 0.01 * expected


def test_coupled_run_with_vegf_vessels_and_pk():
    from synth import make_maps

    n = 10
    cfg = Pm.Config(n, n, n, n_drugs=3, seed=4, vegf=1, vessel_interval=2, pk_model=(0, 2, 1),
                    V_high=5e-5, beta_birth=0.5, p_death=0.5)
    maps = make_maps(n, n, n, corr_len=2.0, seed=4)
    sim = M.OracleSim(cfg, maps.p_cell, maps.perf, maps.p_vessel)
    sim.step(4)
    assert np.all(sim.V >= 0) and sim.V.max() > 0
    h = sim.history
    assert h[0].vessel_births == h[0].vessel_deaths == 0          # step 0: no vascular update
    assert sum(x.vessel_births + x.vessel_deaths for x in h) > 0
    assert all(x.vegf is not None and x.vegf.converged for x in h)
