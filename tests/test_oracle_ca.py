"""Pins for the oracle's cellular-automaton update.

* a separately written brute-force sweep (colour by colour, walking the
  lattice with stride 3) with kill probabilities forced to 0 or 1, run
  exhaustively over one- and two-parent placements and over random
  occupancies;
* invariants: cell balance, daughters only on free sites, blocked cells only
  where no neighbour is free at their turn;
* independence from the order inside a colour;
* kill frequencies against I(x; 1, b) = 1 - (1 - x)^b (Eq. 1 with a = 1).
"""

import itertools
import math

import numpy as np
import pytest

from oracle import params as Pm
from oracle.ca import ca_update

CANCER = (Pm.PROLIF, Pm.QUIESC)
FREE = (Pm.EMPTY, Pm.DEAD)


def brute_force(state, phi, K, kill, shape):
    """Sequential reference: ``kill(x, y, z)`` -> bool decides death."""
    nz, ny, nx = shape
    st = state.copy()
    st[st == Pm.DEAD] = Pm.EMPTY
    committed = {(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)
                 if st[z, y, x] in CANCER and phi[z, y, x] >= 1.0}
    counts = dict(kills=0, divisions=0, blocked=0)
    for cz in range(3):
        for cy in range(3):
            for cx in range(3):
                for z in range(cz, nz, 3):
                    for y in range(cy, ny, 3):
                        for x in range(cx, nx, 3):
                            if (x, y, z) not in committed:
                                continue
                            if kill(x, y, z):
                                st[z, y, x] = Pm.DEAD
                                counts["kills"] += 1
                                continue
                            options = []
                            for rank, (dz, dy, dx) in enumerate(
                                    o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)):
                                xx, yy, zz = x + dx, y + dy, z + dz
                                if 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz and st[zz, yy, xx] in FREE:
                                    options.append((K[zz, yy, xx], -rank, (zz, yy, xx)))
                            if options:
                                target = max(options)[2]
                                st[target] = Pm.PROLIF
                                st[z, y, x] = Pm.PROLIF
                                counts["divisions"] += 1
                            else:
                                st[z, y, x] = Pm.QUIESC
                                counts["blocked"] += 1
    return st, counts


def run_oracle(state, phi, K, G_level, shape, precision="f64"):
    nz, ny, nx = shape
    cfg = Pm.Config(nx=nx, ny=ny, nz=nz, n_drugs=1, precision=precision, seed=3)
    G = [np.full(shape, G_level)]
    zeros = np.zeros(shape)
    return ca_update(state, phi, zeros, zeros, K, G, cfg, step=5)


def check_against_brute(state, phi, K, G_level, shape):
    kill = (lambda x, y, z: True) if G_level >= 1.0 else (lambda x, y, z: False)
    ref_state, counts = brute_force(state, phi, K, kill, shape)
    st, ph, pp, vv, stats = run_oracle(state, phi, K, G_level, shape)
    assert np.array_equal(st, ref_state)
    assert (stats.kills, stats.divisions, stats.blocked) == (counts["kills"], counts["divisions"], counts["blocked"])
    # resets: every site that divided or received a daughter has phi = 0
    changed = (st == Pm.PROLIF) & ((state != Pm.PROLIF) | (phi >= 1.0))
    assert np.all(ph[changed] == 0.0)
    return st, stats


@pytest.mark.parametrize("n", [3, 4])
@pytest.mark.parametrize("G_level", [0.0, 1.0])
def test_single_parent_exhaustive(n, G_level, rng):
    shape = (n, n, n)
    for site in range(n ** 3):
        z, rem = divmod(site, n * n)
        y, x = divmod(rem, n)
        for background in range(3):
            state = np.zeros(shape, dtype=np.uint8)
            if background:
                state[rng.random(shape) < 0.5] = Pm.VESSEL
                state[rng.random(shape) < 0.2] = Pm.DEAD
            state[z, y, x] = Pm.PROLIF
            phi = np.zeros(shape)
            phi[z, y, x] = 1.0
            K = rng.integers(0, 4, shape).astype(np.float64)   # many ties
            check_against_brute(state, phi, K, G_level, shape)


def test_two_parents_exhaustive(rng):
    n = 3
    shape = (n, n, n)
    for a, b in itertools.combinations(range(n ** 3), 2):
        state = np.zeros(shape, dtype=np.uint8)
        phi = np.zeros(shape)
        for s in (a, b):
            z, rem = divmod(s, n * n)
            y, x = divmod(rem, n)
            state[z, y, x] = Pm.PROLIF
            phi[z, y, x] = 1.0 + rng.random()
        K = rng.integers(0, 3, shape).astype(np.float64)
        check_against_brute(state, phi, K, 0.0, shape)


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 4, 6), (6, 6, 6), (3, 5, 7)])
def test_random_occupancies(shape, rng):
    for trial in range(150):
        u = rng.random(shape)
        state = np.full(shape, Pm.EMPTY, dtype=np.uint8)
        state[u < 0.55] = Pm.PROLIF
        state[u < 0.1] = Pm.QUIESC
        state[u < 0.05] = Pm.VESSEL
        state[(u > 0.9) & (u < 0.95)] = Pm.DEAD
        state[u > 0.97] = Pm.STROMA
        phi = rng.random(shape) * 1.5
        K = rng.integers(0, 5, shape).astype(np.float64) if trial % 2 else rng.random(shape)
        st, stats = check_against_brute(state, phi, K, 1.0 if trial % 5 == 0 else 0.0, shape)
        # balance of cancer cells (DEAD sites are cleared before the sweep)
        before = np.isin(state, CANCER).sum()
        after = np.isin(st, CANCER).sum()
        assert after - before == stats.divisions - stats.kills
        # daughters land only on sites that were free (or freed by a kill this sweep)
        new_cells = np.isin(st, CANCER) & ~np.isin(state, CANCER)
        assert np.all(np.isin(state[new_cells], FREE))
        # non-cancer occupants are never touched
        fixed = np.isin(state, (Pm.VESSEL, Pm.STROMA))
        assert np.array_equal(st[fixed], state[fixed])


def test_blocked_only_without_free_neighbour():
    shape = (5, 5, 5)
    state = np.full(shape, Pm.STROMA, dtype=np.uint8)
    state[2, 2, 2] = Pm.PROLIF
    phi = np.zeros(shape)
    phi[2, 2, 2] = 1.2
    K = np.ones(shape)
    st, ph, _, _, stats = run_oracle(state, phi, K, 0.0, shape)
    assert stats.blocked == 1 and st[2, 2, 2] == Pm.QUIESC and ph[2, 2, 2] == 0.0
    state[1, 3, 2] = Pm.DEAD                 # one free (dead) neighbour
    st, ph, _, _, stats = run_oracle(state, phi, K, 0.0, shape)
    assert stats.divisions == 1 and st[1, 3, 2] == Pm.PROLIF and st[2, 2, 2] == Pm.PROLIF


def test_argmax_prefers_highest_oxygen_then_first_in_order():
    shape = (3, 3, 3)
    state = np.zeros(shape, dtype=np.uint8)
    state[1, 1, 1] = Pm.PROLIF
    phi = np.zeros(shape)
    phi[1, 1, 1] = 1.0
    K = np.zeros(shape)
    K[2, 0, 1] = 5.0
    K[0, 2, 2] = 5.0              # equal maximum, earlier in (dz, dy, dx) order
    st, *_ = run_oracle(state, phi, K, 0.0, shape)
    assert st[0, 2, 2] == Pm.PROLIF and st[2, 0, 1] == Pm.EMPTY
    K[2, 0, 1] = 5.5
    st, *_ = run_oracle(state, phi, K, 0.0, shape)
    assert st[2, 0, 1] == Pm.PROLIF and st[0, 2, 2] == Pm.EMPTY


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_in_colour_order_irrelevant(precision, rng):
    shape = (9, 10, 11)
    u = rng.random(shape)
    state = np.where(u < 0.6, Pm.PROLIF, Pm.EMPTY).astype(np.uint8)
    state[u < 0.08] = Pm.VESSEL
    phi = rng.random(shape) * 1.3
    K = rng.random(shape)
    nz, ny, nx = shape
    cfg = Pm.Config(nx=nx, ny=ny, nz=nz, n_drugs=2, precision=precision, seed=11, kill_b=(2, 1, 1))
    G = [rng.random(shape) * 0.6, rng.random(shape) * 0.3]
    zeros = np.zeros(shape)
    base = ca_update(state, phi, zeros, zeros, K, G, cfg, 3)
    perm_rng = np.random.default_rng(1)
    for order in (lambda s: s[::-1], lambda s: list(perm_rng.permutation(s))):
        other = ca_update(state, phi, zeros, zeros, K, G, cfg, 3, order=order)
        assert np.array_equal(base[0], other[0])
        assert np.array_equal(base[1], other[1])
        assert base[4] == other[4]


@pytest.mark.parametrize("x,b,n_drugs", [(0.3, 1, 1), (0.3, 2, 1), (0.5, 3, 1), (0.2, 1, 2)])
def test_kill_frequency_matches_incomplete_beta(x, b, n_drugs):
    n = 36
    shape = (n, n, n)
    state = np.full(shape, Pm.PROLIF, dtype=np.uint8)
    phi = np.ones(shape)
    K = np.zeros(shape)
    cfg = Pm.Config(nx=n, ny=n, nz=n, n_drugs=n_drugs, seed=77, kill_b=(b, b, b))
    G = [np.full(shape, x)] * n_drugs
    zeros = np.zeros(shape)
    st, _, _, _, stats = ca_update(state, phi, zeros, zeros, K, G, cfg, 0)
    p = 1.0 - ((1.0 - x) ** b) ** n_drugs
    frac = stats.kills / n ** 3
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / n ** 3), (frac, p)
