"""The stochastic cellular-automaton update of cancer cells.

Sections 2.2.1 and 2.5 of the paper.  A cancer cell whose cycle clock has
reached phi >= 1 is committed.  It is first killed by the drugs with the
probability given by the regularised incomplete beta function I(x; 1, b)
(Eq. 1); otherwise a daughter is placed on the free Moore neighbour with the
highest oxygen K, and phi, P and Vc of parent and daughter are reset to zero.
If no neighbour is free, only the parent's cycle clock is reset.

Readings used (the paper does not fix them):

* 3-D Moore neighbourhood (26 sites), clipped at the lattice boundary.
* With a = 1 the incomplete beta function has the closed form
  I(x; 1, b) = 1 - (1 - x)^b; b is a positive integer and the power is taken
  by repeated multiplication.  x = G_d / max G_{d,0} clamped to [0, 1].
* Several drugs act independently: P_kill = 1 - prod_d (1 - I_d).
* Sweep order: colour c = (x mod 3) + 3 (y mod 3) + 9 (z mod 3), c = 0..26;
  later colours see the daughters and deaths of earlier colours (a
  Gauss-Seidel sweep).  Two sites of one colour are >= 3 apart along some
  axis, so their closed neighbourhoods are disjoint and the order inside a
  colour does not matter.  This replaces the paper's cross-process "higher
  phi wins" rule (Algorithm 2).
* Argmax over free neighbours in the fixed order dz, dy, dx in (-1, 0, 1),
  lexicographic; on equal K the first neighbour in that order wins.
* Free = EMPTY or DEAD.  A killed cell becomes DEAD (acts as EMPTY) and is
  cleared to EMPTY at the start of the next update.  A blocked cell becomes
  QUIESC; a cell that divides (and its daughter) is PROLIF.
* Resets follow the prose (phi = P = Vc = 0 for parent and daughter); the
  copy-the-parent line of Algorithm 2 is not used.
* Decision arithmetic is done in the storage precision of the fields
  (float32 or float64), with IEEE round-to-nearest basic operations only.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import params as Pm
from .philox import site_uniform

NEIGHBOUR_OFFSETS = tuple((dz, dy, dx)
                          for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                          if (dz, dy, dx) != (0, 0, 0))


@dataclasses.dataclass
class CAStats:
    committed: int = 0
    kills: int = 0
    divisions: int = 0
    blocked: int = 0


def colour_of(x, y, z):
    return (x % 3) + 3 * (y % 3) + 9 * (z % 3)


def survival_probability(G_site, cfg: Pm.Config, dtype):
    """prod_d (1 - x_d)^{b_d}, x_d = clamp(G_d / max G_{d,0}, 0, 1), in ``dtype``."""
    one = dtype(1.0)
    survive = one
    for d in range(cfg.n_drugs):
        x = dtype(G_site[d]) / dtype(cfg.dose_peak[d])
        if x > one:
            x = one
        if x < dtype(0.0):
            x = dtype(0.0)
        f = one - x
        for _ in range(int(cfg.kill_b[d])):
            survive = dtype(survive * f)
    return survive


def ca_update(state, phi, P, Vc, K, G, cfg: Pm.Config, step: int, order=None):
    """One CA update.  Returns (state, phi, P, Vc, CAStats); inputs are not modified.

    ``G`` is a sequence of n_drugs arrays.  ``order``, if given, is a callable
    that permutes the committed sites of one colour (used by tests to show
    that the in-colour order is irrelevant).
    """
    dtype = np.float32 if cfg.precision == "f32" else np.float64
    nz, ny, nx = state.shape
    st = np.array(state, dtype=np.uint8, copy=True).reshape(-1)
    ph = np.array(phi, dtype=np.float64, copy=True).reshape(-1)
    pp = np.array(P, dtype=np.float64, copy=True).reshape(-1)
    vv = np.array(Vc, dtype=np.float64, copy=True).reshape(-1)
    Kf = np.asarray(K, dtype=dtype).reshape(-1)
    Gf = [np.asarray(g, dtype=dtype).reshape(-1) for g in G]

    st[st == Pm.DEAD] = Pm.EMPTY
    committed = np.flatnonzero(np.isin(st, Pm.CANCER_STATES) & (ph.astype(dtype) >= dtype(1.0)))
    stats = CAStats(committed=int(committed.size))
    u_all = site_uniform(cfg.seed, committed, step, Pm.PURPOSE_KILL).astype(dtype)
    u_of = dict(zip(committed.tolist(), u_all.tolist()))

    zs, rem = np.divmod(committed, nx * ny)
    ys, xs = np.divmod(rem, nx)
    colours = colour_of(xs, ys, zs)

    for c in range(27):
        sites = committed[colours == c].tolist()
        if order is not None:
            sites = order(sites)
        for s in sites:
            z, rem_s = divmod(s, nx * ny)
            y, x = divmod(rem_s, nx)
            u = dtype(u_of[s])
            survive = survival_probability([g[s] for g in Gf], cfg, dtype)
            p_kill = dtype(dtype(1.0) - survive)
            if u < p_kill:
                st[s] = Pm.DEAD
                ph[s] = pp[s] = vv[s] = 0
                stats.kills += 1
                continue
            best = -1
            best_K = None
            for dz, dy, dx in NEIGHBOUR_OFFSETS:
                xx, yy, zz = x + dx, y + dy, z + dz
                if not (0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz):
                    continue
                n = xx + nx * (yy + ny * zz)
                if st[n] in Pm.FREE_STATES and (best < 0 or Kf[n] > best_K):
                    best, best_K = n, Kf[n]
            if best >= 0:
                st[best] = Pm.PROLIF
                st[s] = Pm.PROLIF
                ph[s] = pp[s] = vv[s] = 0
                ph[best] = pp[best] = vv[best] = 0
                stats.divisions += 1
            else:
                st[s] = Pm.QUIESC
                ph[s] = 0
                stats.blocked += 1
    shape = (nz, ny, nx)
    return st.reshape(shape), ph.reshape(shape), pp.reshape(shape), vv.reshape(shape), stats
