"""The synchronous cellular-automaton update with the "higher phi wins" rule.

Section 2.5 says the updates of proliferation-ready cells are asynchronous in
the sense that a cell's new state does not enter its neighbours' decisions;
Algorithm 2 resolves two parents placing a daughter on the same site by
giving the site to the parent with the higher cycle clock phi.  Written out:

  1. DEAD sites become EMPTY; every cancer cell with phi >= 1 is committed.
  2. Each committed cell is killed with probability 1 - prod_d (1 - x_d)^{b_d}
     (Eq. 1, the same Philox draw as the colour sweep in ca.py).
  3. Each survivor picks the free Moore neighbour with the highest K in the
     lattice as it was before the update (kills and daughters of this update
     are not seen; first in dz, dy, dx order on equal K).
  4. A site picked by several parents goes to the one with the highest phi;
     on equal phi to the one with the lowest site index (reading: the paper
     does not break ties).
  5. Winners divide (parent and daughter PROLIF, phi = P = Vc = 0); a parent
     with no free neighbour, or that lost its site, is blocked (QUIESC,
     phi = 0); killed cells become DEAD with phi = P = Vc = 0.

Readings shared with ca.py: Moore neighbourhood clipped at the boundary,
free = EMPTY or DEAD, resets by the prose rather than Algorithm 2's copy of
the parent, decisions in the storage precision.  Test infrastructure only.
"""

from __future__ import annotations

import numpy as np

from . import params as Pm
from .ca import NEIGHBOUR_OFFSETS, CAStats, survival_probability
from .philox import site_uniform


def ca_update_sync(state, phi, P, Vc, K, G, cfg: Pm.Config, step: int):
    """One synchronous CA update.  Returns (state, phi, P, Vc, CAStats)."""
    dtype = np.float32 if cfg.precision == "f32" else np.float64
    nz, ny, nx = state.shape
    st = np.array(state, dtype=np.uint8, copy=True).reshape(-1)
    ph = np.array(phi, dtype=np.float64, copy=True).reshape(-1)
    pp = np.array(P, dtype=np.float64, copy=True).reshape(-1)
    vv = np.array(Vc, dtype=np.float64, copy=True).reshape(-1)
    Kf = np.asarray(K, dtype=dtype).reshape(-1)
    Gf = [np.asarray(g, dtype=dtype).reshape(-1) for g in G]

    st[st == Pm.DEAD] = Pm.EMPTY
    old = st.copy()                                   # the lattice every decision reads
    committed = np.flatnonzero(np.isin(old, Pm.CANCER_STATES) & (ph.astype(dtype) >= dtype(1.0)))
    stats = CAStats(committed=int(committed.size))
    u_all = site_uniform(cfg.seed, committed, step, Pm.PURPOSE_KILL).astype(dtype)

    killed, target = [], {}
    for s, u in zip(committed.tolist(), u_all.tolist()):
        p_kill = dtype(dtype(1.0) - survival_probability([g[s] for g in Gf], cfg, dtype))
        if dtype(u) < p_kill:
            killed.append(s)
            continue
        z, rem = divmod(s, nx * ny)
        y, x = divmod(rem, nx)
        best, best_K = -1, None
        for dz, dy, dx in NEIGHBOUR_OFFSETS:
            xx, yy, zz = x + dx, y + dy, z + dz
            if 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz:
                n = xx + nx * (yy + ny * zz)
                if old[n] in Pm.FREE_STATES and (best < 0 or Kf[n] > best_K):
                    best, best_K = n, Kf[n]
        target[s] = best

    # the winner of each picked site: highest phi (storage precision), then lowest index
    winner = {}
    for s, t in target.items():
        if t < 0:
            continue
        key = (-float(dtype(ph[s])), s)
        if t not in winner or key < winner[t][0]:
            winner[t] = (key, s)

    for s in killed:
        st[s] = Pm.DEAD
        ph[s] = pp[s] = vv[s] = 0
        stats.kills += 1
    for s, t in target.items():
        if t >= 0 and winner[t][1] == s:
            st[s] = st[t] = Pm.PROLIF
            ph[s] = pp[s] = vv[s] = 0
            ph[t] = pp[t] = vv[t] = 0
            stats.divisions += 1
        else:
            st[s] = Pm.QUIESC
            ph[s] = 0
            stats.blocked += 1
    shape = (nz, ny, nx)
    return st.reshape(shape), ph.reshape(shape), pp.reshape(shape), vv.reshape(shape), stats
