"""Shared set-up for the GPU parity tests: the same seeded inputs for both sides."""

import numpy as np

from oracle import params as Pm
from paper_2105_00448_gb300 import hca
from synth import make_maps


def make_pair(shape, precision="f64", corr_len=3.0, threads=0, **params):
    """A library handle and the oracle config for one (nz, ny, nx) lattice."""
    nz, ny, nx = shape
    maps = make_maps(nx, ny, nz, corr_len=corr_len, seed=params.get("seed", 0))
    sim = hca.Sim.create(nx, ny, nz, maps.p_cell, maps.perf, maps.p_vessel, precision=precision,
                         threads_per_block=threads, **params)
    # library-only settings (precision scheme, tiling) have no oracle counterpart
    oracle_params = {k: v for k, v in params.items() if k in Pm.Config.__dataclass_fields__}
    cfg = Pm.Config(nx=nx, ny=ny, nz=nz, precision=precision, **oracle_params)
    return sim, cfg, maps


def random_states(shape, rng, p_vessel=0.1, p_cancer=0.45, p_stroma=0.03, p_dead=0.04):
    u = rng.random(shape)
    st = np.full(shape, Pm.EMPTY, dtype=np.uint8)
    edges = np.cumsum([p_vessel, p_cancer, p_stroma, p_dead])
    st[u < edges[3]] = Pm.DEAD
    st[u < edges[2]] = Pm.STROMA
    st[u < edges[1]] = Pm.PROLIF
    st[u < edges[0]] = Pm.VESSEL
    q = rng.random(shape)
    st[(st == Pm.PROLIF) & (q < 0.3)] = Pm.QUIESC
    return st


def operator_scale(coupling, reaction, u):
    """Size of the terms of (A u)_i, the yardstick for rounding differences."""
    return float(np.max(np.abs(reaction) * np.abs(u)) + coupling * 7.0 * np.max(np.abs(u)))


def oracle_trajectory(args):
    """One oracle replicate of the coupled run, step by step (for a spawn
    process pool): (seed, edge, steps, corr_len, params) -> int64 array
    (steps, 8): the count of each state code after every step, then that
    step's kills and divisions."""
    seed, edge, steps, corr_len, params = args
    from oracle.model import OracleSim

    cfg = Pm.Config(nx=edge, ny=edge, nz=edge, seed=seed, **params)
    maps = make_maps(edge, edge, edge, corr_len=corr_len, seed=seed)
    sim = OracleSim(cfg, maps.p_cell, maps.perf, maps.p_vessel)
    out = np.zeros((steps, 8), dtype=np.int64)
    for t in range(steps):
        sim.step(1)
        h = sim.history[-1]
        out[t, :6] = np.bincount(sim.state.reshape(-1), minlength=6)
        out[t, 6], out[t, 7] = h.kills, h.divisions
    return out
