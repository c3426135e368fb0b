"""The oracle's call-name veneer (oracle.api) returns what OracleSim holds,
packs fields like the library (increasing bit order) and rejects what the
library rejects."""

import numpy as np
import pytest

from oracle import api
from oracle import params as Pm
from oracle.model import OracleSim
from synth import make_maps


def test_api_matches_the_simulation():
    n = 8
    cfg = Pm.Config(n, n, n, n_drugs=2, seed=3)
    m = make_maps(n, n, n, corr_len=2.0, seed=3)
    h = api.oracle_create(cfg, m.p_cell, m.perf, m.p_vessel)
    sim = OracleSim(cfg, m.p_cell, m.perf, m.p_vessel)
    api.oracle_step(h, 2)
    sim.step(2)
    assert np.array_equal(api.oracle_read_states(h, 0), sim.state.reshape(-1))
    packed = api.oracle_read_fields(h, 0, api.FIELD_O2 | api.FIELD_DRUG[1] | api.FIELD_PHI)
    ref = np.concatenate([sim.K.reshape(-1), sim.G[1].reshape(-1), sim.phi.reshape(-1)])
    assert np.array_equal(packed, ref)
    st = api.oracle_get_stats(h, 0)
    assert st["step"] == 2 and st["counts"] == [int(c) for c in sim.history[-1].counts]
    assert len(st["drug_iterations"]) == 2
    with pytest.raises(ValueError):
        api.oracle_read_fields(h, 0, api.FIELD_DRUG[2])      # two drugs only
    with pytest.raises(ValueError):
        api.oracle_read_fields(h, 0, 1 << 9)
    api.oracle_destroy(h)
    assert h.sims == []


def test_batch_replicates_are_independent():
    cfgs, maps = [], []
    for r, n in enumerate((6, 8)):
        cfgs.append(Pm.Config(n, n, n, n_drugs=1, seed=10 + r))
        maps.append(make_maps(n, n, n, corr_len=2.0, seed=10 + r))
    h = api.oracle_create_batch(cfgs, [m.p_cell for m in maps], [m.perf for m in maps], [m.p_vessel for m in maps])
    api.oracle_step(h, 1)
    for r in range(2):
        alone = api.oracle_create(cfgs[r], maps[r].p_cell, maps[r].perf, maps[r].p_vessel)
        api.oracle_step(alone, 1)
        assert np.array_equal(api.oracle_read_states(h, r), api.oracle_read_states(alone, 0))
