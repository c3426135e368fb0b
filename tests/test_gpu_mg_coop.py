"""The coarse levels of the V-cycle in one cooperative launch (grid barriers
between levels, the single-block levels in shared memory) against one launch
per level (HCA_MG_COOP=0, read at handle creation): both run the same per-site
arithmetic in the same order, so z = M r, whole solves and coupled steps must
agree bit for bit, in FP64 and FP32, for single lattices and batches.  The
library uses the cooperative launch from host-driven loops (the coupled runs
here set HCA_NO_GRAPH=1) and per-level launches inside captured step graphs
(HCA_MG_COOP_GRAPH=2 captures the cooperative launch for the levels below
2^18 sites).  The V-cycle itself is compared with the oracle in
test_gpu_mg.py.
"""

import os

import numpy as np
import pytest

from gpu_helpers import make_pair, random_states
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu

# grid-kernel coarse levels (row-vector and per-site forms), a flat lattice,
# odd extents, and a lattice whose level 1 is already a single-block level
SHAPES = [(24, 40, 56), (64, 64, 64), (1, 48, 70), (17, 23, 31), (40, 36, 44), (16, 16, 16)]


def _with_coop(flag, fn, no_graph=False):
    old = {k: os.environ.get(k) for k in ("HCA_MG_COOP", "HCA_NO_GRAPH")}
    os.environ["HCA_MG_COOP"] = "1" if flag else "0"
    if no_graph:
        os.environ["HCA_NO_GRAPH"] = "1"
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_vcycle_coop_equals_per_level_launches(shape, which, precision):
    rng = np.random.default_rng(31)
    st = random_states(shape, rng)
    K = rng.uniform(0.0, 20.0, shape)
    r = rng.standard_normal(shape)

    def run():
        sim, _, _ = make_pair(shape, precision, seed=2, n_drugs=1, preconditioner=hca.HCA_PC_MG, picard_maxit=1)
        sim.set_states(st)
        sim.set_field(hca.FIELD_O2, K)
        z = sim.apply_preconditioner(which, r)
        sim.close()
        return z

    z_coop = _with_coop(True, run)
    z_levels = _with_coop(False, run)
    assert np.array_equal(z_coop, z_levels)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_coupled_steps_coop_equal_per_level_launches(precision):
    n = 48

    def run():
        maps = make_maps(n, n, n, corr_len=4.0, seed=5)
        sim = hca.Sim.create(n, n, n, maps.p_cell, maps.perf, maps.p_vessel, precision=precision, n_drugs=2,
                             seed=5, preconditioner=hca.HCA_PC_MG)
        sim.step(3)
        out = (sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG0), sim.field(hca.FIELD_DRUG1),
               sim.stats())
        sim.close()
        return out

    a = _with_coop(True, run, no_graph=True)
    b = _with_coop(False, run, no_graph=True)
    assert np.array_equal(a[0], b[0])
    for k in (1, 2, 3):
        assert np.array_equal(a[k], b[k])
    assert a[4]["o2_iterations"] == b[4]["o2_iterations"]
    assert a[4]["drug_iterations"] == b[4]["drug_iterations"]


def test_batch_coop_equals_per_level_launches():
    sizes = [(20, 24, 28), (33, 17, 40), (48, 48, 48)]

    def run():
        cfgs, maps = [], []
        for i, (nz, ny, nx) in enumerate(sizes):
            m = make_maps(nx, ny, nz, corr_len=3.0, seed=10 + i)
            maps.append((m.p_cell, m.perf, m.p_vessel))
            cfgs.append(hca.make_config(nx, ny, nz, precision="f32", n_drugs=1, seed=10 + i,
                                        preconditioner=hca.HCA_PC_MG))
        sim = hca.Sim(cfgs, maps, batch=True)
        sim.step(2)
        out = [(sim.states(i), sim.field(hca.FIELD_O2, i), sim.field(hca.FIELD_DRUG0, i)) for i in range(len(sizes))]
        sim.close()
        return out

    a = _with_coop(True, run, no_graph=True)
    b = _with_coop(False, run, no_graph=True)
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("n", [48, 160])
def test_graph_steps_with_coop_tail_equal_per_level_launches(n):
    """Captured step graphs with HCA_MG_COOP_GRAPH=2: at 160^3 level 1
    (80^3 sites) keeps its per-level kernels and the cooperative launch
    starts at level 2; at 48^3 it starts at level 1.  Both give the
    per-level launches' bits."""

    def run():
        maps = make_maps(n, n, n, corr_len=4.0, seed=7)
        sim = hca.Sim.create(n, n, n, maps.p_cell, maps.perf, maps.p_vessel, precision="f32", n_drugs=2,
                             seed=7, preconditioner=hca.HCA_PC_MG)
        sim.step(2)
        out = (sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_DRUG1), sim.stats())
        sim.close()
        return out

    os.environ["HCA_MG_COOP_GRAPH"] = "2"
    try:
        a = _with_coop(True, run)
    finally:
        os.environ.pop("HCA_MG_COOP_GRAPH", None)
    b = _with_coop(False, run)
    for k in range(3):
        assert np.array_equal(a[k], b[k])
    assert a[3]["drug_iterations"] == b[3]["drug_iterations"]
