"""The 27 colour sweeps of the CA update in one cooperative launch (a grid
barrier between colours) against one launch per colour (HCA_CA_COOP=0, read
at handle creation): the per-cell step is the same and colour c + 1 starts
only after colour c is complete in both forms, so coupled runs must agree bit
for bit (states, fields, kills, divisions), for FP64 and FP32, single
lattices and batches, from the step graph and from the host loop.  The CA
itself is compared with the oracle in test_gpu_parity.py.
"""

import os

import numpy as np
import pytest

from gpu_helpers import make_pair
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu


def _with(env, fn):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("no_graph", ["0", "1"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_colour_sweeps_in_one_launch_equal_per_colour(precision, no_graph):
    shape = (30, 34, 41)

    def run():
        sim, _, _ = make_pair(shape, precision, seed=12, n_drugs=2, preconditioner=hca.HCA_PC_MG)
        out = []
        for _ in range(4):
            sim.step(1)
            st = sim.stats()
            out.append((sim.states(), sim.field(hca.FIELD_PHI), st["kills"], st["divisions"], st["blocked"]))
        sim.close()
        return out

    a = _with({"HCA_CA_COOP": "1", "HCA_NO_GRAPH": no_graph}, run)
    b = _with({"HCA_CA_COOP": "0", "HCA_NO_GRAPH": no_graph}, run)
    assert sum(x[3] for x in a) > 0
    for x, y in zip(a, b):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2:] == y[2:]


def test_batch_colour_sweeps_in_one_launch_equal_per_colour():
    sizes = [(20, 24, 28), (33, 17, 40), (12, 50, 20)]

    def run():
        cfgs, maps = [], []
        for i, (nz, ny, nx) in enumerate(sizes):
            m = make_maps(nx, ny, nz, corr_len=3.0, seed=20 + i)
            maps.append((m.p_cell, m.perf, m.p_vessel))
            cfgs.append(hca.make_config(nx, ny, nz, precision="f32", n_drugs=1, seed=20 + i))
        sim = hca.Sim(cfgs, maps, batch=True)
        sim.step(3)
        out = [(sim.states(i), sim.stats(i)["kills"], sim.stats(i)["divisions"]) for i in range(len(sizes))]
        sim.close()
        return out

    a = _with({"HCA_CA_COOP": "1"}, run)
    b = _with({"HCA_CA_COOP": "0"}, run)
    for x, y in zip(a, b):
        assert np.array_equal(x[0], y[0]) and x[1:] == y[1:]
