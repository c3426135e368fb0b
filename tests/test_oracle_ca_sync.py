"""The oracle's synchronous CA update (oracle.ca_sync, Section 2.5 with
Algorithm 2's higher-phi rule) pinned by hand-built conflicts, by an
order-based brute force written here, by its equality with the colour sweep
when committed cells are too far apart to interact, and by conservation."""

import numpy as np
import pytest

from oracle import params as Pm
from oracle.ca import NEIGHBOUR_OFFSETS, ca_update, survival_probability
from oracle.ca_sync import ca_update_sync
from oracle.philox import site_uniform


def _line(states, phis, K, G=None, n_drugs=0):
    n = len(states)
    cfg = Pm.Config(n, 1, 1, n_drugs=n_drugs, kill_b=(1, 1, 1))
    st = np.array(states, dtype=np.uint8).reshape(1, 1, n)
    ph = np.array(phis, dtype=np.float64).reshape(1, 1, n)
    z = np.zeros((1, 1, n))
    Gs = [np.array(G, dtype=np.float64).reshape(1, 1, n)] if G is not None else []
    return cfg, st, ph, z, np.array(K, dtype=np.float64).reshape(1, 1, n), Gs


@pytest.mark.parametrize("phiA,phiB,winner", [(1.5, 1.2, 0), (1.2, 1.5, 2), (1.3, 1.3, 0)])
def test_contested_site_goes_to_higher_phi(phiA, phiB, winner):
    E, PR, ST = Pm.EMPTY, Pm.PROLIF, Pm.STROMA
    cfg, st, ph, z, K, G = _line([PR, E, PR], [phiA, 0, phiB], [1, 5, 1])
    s, p, _, _, stats = ca_update_sync(st, ph, z, z, K, G, cfg, 0)
    loser = 2 - winner
    assert s[0, 0, 1] == PR and s[0, 0, winner] == PR and s[0, 0, loser] == Pm.QUIESC
    assert p[0, 0, winner] == 0 and p[0, 0, loser] == 0 and p[0, 0, 1] == 0
    assert (stats.divisions, stats.blocked, stats.kills) == (1, 1, 0)


def test_loser_does_not_fall_back_and_kills_free_nothing():
    E, PR, ST = Pm.EMPTY, Pm.PROLIF, Pm.STROMA
    # B (x=2) prefers x=1 (K 5) over x=3 (K 4) and loses x=1 to A: blocked,
    # where the colour sweep would have sent it to x=3
    cfg, st, ph, z, K, G = _line([PR, E, PR, E], [1.5, 0, 1.2, 0], [1, 5, 1, 4])
    s, *_ = ca_update_sync(st, ph, z, z, K, G, cfg, 0)
    assert list(s.reshape(-1)) == [PR, PR, Pm.QUIESC, E]
    s_gs, *_ = ca_update(st, ph, z, z, K, G, cfg, 0)
    assert list(s_gs.reshape(-1)) == [PR, PR, PR, PR]
    # A (x=0) is killed for sure (G = peak, b = 1); B (x=1) never; B does not
    # see A's site as free in the same update
    cfg, st, ph, z, K, G = _line([PR, PR, ST], [1.1, 1.1, 0], [9, 1, 1], G=[1.0, 0.0, 0.0], n_drugs=1)
    s, _, _, _, stats = ca_update_sync(st, ph, z, z, K, G, cfg, 0)
    assert list(s.reshape(-1)) == [Pm.DEAD, Pm.QUIESC, ST]
    assert (stats.kills, stats.blocked, stats.divisions) == (1, 1, 0)
    s_gs, *_ = ca_update(st, ph, z, z, K, G, cfg, 0)
    assert list(s_gs.reshape(-1)) == [PR, PR, ST]


def _brute_sync(state, phi, K, G, cfg, step, order_rng):
    """Parents visited in a random order; each claim replaces the current one
    when its phi is higher or equal with a lower index; outcomes applied at
    the end."""
    dtype = np.float32 if cfg.precision == "f32" else np.float64
    nz, ny, nx = state.shape
    st = state.reshape(-1).copy()
    st[st == Pm.DEAD] = Pm.EMPTY
    old = st.copy()
    ph = phi.reshape(-1).astype(np.float64).copy()
    sites = [i for i in range(st.size) if old[i] in Pm.CANCER_STATES and dtype(ph[i]) >= 1]
    order_rng.shuffle(sites)
    claims, outcome = {}, {}
    for s in sites:
        u = dtype(site_uniform(cfg.seed, np.array([s], dtype=np.uint64), step, Pm.PURPOSE_KILL)[0])
        if u < dtype(1) - survival_probability([g.reshape(-1)[s] for g in G], cfg, dtype):
            outcome[s] = "kill"
            continue
        z, r = divmod(s, nx * ny)
        y, x = divmod(r, nx)
        cands = []
        for dz, dy, dx in NEIGHBOUR_OFFSETS:
            if 0 <= x + dx < nx and 0 <= y + dy < ny and 0 <= z + dz < nz:
                n = (x + dx) + nx * ((y + dy) + ny * (z + dz))
                if old[n] in Pm.FREE_STATES:
                    cands.append(n)
        if not cands:
            outcome[s] = "block"
            continue
        kv = K.reshape(-1).astype(dtype)
        t = cands[0]
        for n in cands[1:]:
            if kv[n] > kv[t]:
                t = n
        outcome[s] = t
        c = claims.get(t)
        if c is None or dtype(ph[s]) > dtype(ph[c]) or (dtype(ph[s]) == dtype(ph[c]) and s < c):
            claims[t] = s
    for s, o in outcome.items():
        if o == "kill":
            st[s] = Pm.DEAD
        elif o == "block" or claims[o] != s:
            st[s] = Pm.QUIESC
        else:
            st[s] = st[o] = Pm.PROLIF
    return st.reshape(state.shape)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_order_based_brute_force(seed, precision):
    rng = np.random.default_rng(seed)
    shape = (3, 7, 9)
    cfg = Pm.Config(9, 7, 3, n_drugs=2, seed=seed, precision=precision, kill_b=(2, 3, 1))
    u = rng.random(shape)
    st = np.where(u < 0.5, Pm.PROLIF, np.where(u < 0.55, Pm.QUIESC, np.where(u < 0.6, Pm.DEAD,
                  np.where(u < 0.65, Pm.STROMA, Pm.EMPTY)))).astype(np.uint8)
    # quantised phi values so that equal-phi ties occur
    phi = np.round(rng.uniform(0.8, 1.6, shape) * 8) / 8
    K = np.round(rng.uniform(0, 20, shape))
    G = [rng.uniform(0, 0.6, shape) for _ in range(2)]
    ref, *_ = ca_update_sync(st, phi, np.zeros(shape), np.zeros(shape), K, G, cfg, 5)
    for k in range(4):
        got = _brute_sync(st, phi, K, G, cfg, 5, np.random.default_rng(100 + k))
        assert np.array_equal(got, ref)


def test_equals_colour_sweep_when_cells_do_not_interact():
    """Committed cells at Chebyshev distance >= 3 have disjoint closed
    neighbourhoods: both update rules give the same lattice."""
    rng = np.random.default_rng(4)
    shape = (6, 9, 12)
    cfg = Pm.Config(12, 9, 6, n_drugs=1, seed=3)
    st = np.where(rng.random(shape) < 0.5, Pm.STROMA, Pm.EMPTY).astype(np.uint8)
    phi = np.zeros(shape)
    for z in range(0, 6, 3):
        for y in range(0, 9, 3):
            for x in range(0, 12, 3):
                st[z, y, x] = Pm.PROLIF
                phi[z, y, x] = rng.uniform(1.0, 1.5)
    K = rng.uniform(0, 20, shape)
    G = [rng.uniform(0, 0.7, shape)]
    z0 = np.zeros(shape)
    a = ca_update(st, phi, z0, z0, K, G, cfg, 2)
    b = ca_update_sync(st, phi, z0, z0, K, G, cfg, 2)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert (a[4].kills, a[4].divisions, a[4].blocked) == (b[4].kills, b[4].divisions, b[4].blocked)


def test_conservation():
    rng = np.random.default_rng(9)
    shape = (5, 8, 8)
    cfg = Pm.Config(8, 8, 5, n_drugs=1, seed=9)
    st = np.where(rng.random(shape) < 0.6, Pm.PROLIF, Pm.EMPTY).astype(np.uint8)
    phi = rng.uniform(0.5, 1.5, shape)
    K = rng.uniform(0, 20, shape)
    G = [rng.uniform(0, 0.5, shape)]
    z0 = np.zeros(shape)
    s, p, _, _, stats = ca_update_sync(st, phi, z0, z0, K, G, cfg, 1)
    live = lambda a: int(np.isin(a, Pm.CANCER_STATES).sum())
    assert live(s) == live(st) - stats.kills + stats.divisions
    assert stats.committed == stats.kills + stats.divisions + stats.blocked
    new_cells = (~np.isin(st, Pm.CANCER_STATES)) & np.isin(s, Pm.CANCER_STATES)
    assert int(new_cells.sum()) == stats.divisions
