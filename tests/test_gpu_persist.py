"""Alternative launch forms of one FP32 lattice's kernels against each other,
bit for bit (the form is read at handle creation):

* persistent row kernels (CG pass A, pass B and the lattice post-sweep of the
  V-cycle, one row per warp) against the one-block-per-chunk form
  (HCA_PERSIST=0): every row is computed by the same code and its sum goes to
  the same chunk slot, and each chunk is summed in the same fixed tree.
  Lattices: one, two and four groups per lane, chunks of 8 and 32 rows,
  ragged rows, both preconditioners;
* the plane-marching multigrid sweeps (lattice pre-sweeps with TMA-staged or
  register-prefetched planes, HCA_MG_ZMARCH; grid-level sweeps,
  HCA_MG_ZLEVELS) against the row forms: the same arithmetic per site in the
  same order.

Their parity with the oracle is checked in test_gpu_bench_instances.py and
test_gpu_mg.py.
"""

import os

import numpy as np
import pytest

from gpu_helpers import make_pair
from paper_2105_00448_gb300 import hca

pytestmark = pytest.mark.gpu

SHAPES = [(24, 32, 160), (16, 16, 256), (32, 64, 128), (13, 24, 130), (8, 20, 300), (64, 64, 64)]


def _with_persist(flag, fn):
    old = os.environ.get("HCA_PERSIST")
    os.environ["HCA_PERSIST"] = "1" if flag else "0"
    try:
        return fn()
    finally:
        if old is None:
            del os.environ["HCA_PERSIST"]
        else:
            os.environ["HCA_PERSIST"] = old


@pytest.mark.parametrize("pc", [hca.HCA_PC_MG, hca.HCA_PC_JACOBI], ids=["mg", "jacobi"])
@pytest.mark.parametrize("shape", SHAPES)
def test_persistent_rows_equal_block_per_chunk(shape, pc):
    def run():
        sim, _, _ = make_pair(shape, "f32", seed=9, n_drugs=2, preconditioner=pc)
        sim.step(3)
        out = (sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_O2_LO), sim.field(hca.FIELD_DRUG0),
               sim.field(hca.FIELD_DRUG1), sim.stats())
        sim.close()
        return out

    a = _with_persist(True, run)
    b = _with_persist(False, run)
    for u, v in zip(a[:5], b[:5]):
        assert np.array_equal(u, v)
    assert a[5]["o2_iterations"] == b[5]["o2_iterations"]
    assert a[5]["drug_iterations"] == b[5]["drug_iterations"]
    assert a[5]["o2_rel_residual"] == b[5]["o2_rel_residual"]


ZM_SHAPES = [(24, 32, 160), (13, 24, 130), (8, 20, 300), (64, 64, 64), (5, 17, 36), (3, 40, 260)]


@pytest.mark.parametrize("waves", ["1", "8", "0.05"], ids=["wave", "thin-slabs", "one-slab"])
@pytest.mark.parametrize("mode", ["1", "2"], ids=["registers", "tma"])
@pytest.mark.parametrize("shape", ZM_SHAPES)
def test_plane_marching_presweeps_equal_row_form(shape, mode, waves, monkeypatch):
    """The lattice pre-sweeps in plane-marching form (tiles of 32 x 16 sites,
    slabs of planes; planes prefetched into registers with the halo in shared
    memory, or staged in shared memory by TMA tensor copies) give the row
    form's bits: one V-cycle z = M r on a random r, and two coupled steps.
    Ragged tiles in x and y, slabs of one plane up to the whole lattice."""
    rng = np.random.default_rng(21)
    r = rng.standard_normal(shape).astype(np.float32)
    out = []
    for zm in ("0", mode):
        monkeypatch.setenv("HCA_MG_ZMARCH", zm)
        monkeypatch.setenv("HCA_MG_ZM_WAVES", waves)
        sim, _, _ = make_pair(shape, "f32", seed=17, n_drugs=2, preconditioner=hca.HCA_PC_MG)
        z = [sim.apply_preconditioner(w, r) for w in (0, 1)]
        sim.step(2)
        out.append((z, sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_O2_LO),
                    sim.field(hca.FIELD_DRUG0), sim.field(hca.FIELD_DRUG1), sim.stats()))
        sim.close()
    a, b = out
    for u, v in zip(a[0], b[0]):
        assert np.isfinite(u).all() and np.abs(u).max() > 0
        assert np.array_equal(u, v)
    for u, v in zip(a[1:6], b[1:6]):
        assert np.array_equal(u, v)
    assert a[6]["o2_iterations"] == b[6]["o2_iterations"]
    assert a[6]["drug_iterations"] == b[6]["drug_iterations"]


@pytest.mark.parametrize("waves", ["1", "0.05"], ids=["wave", "one-slab"])
@pytest.mark.parametrize("shape", [(64, 64, 64), (24, 40, 136), (9, 36, 72)])
def test_plane_marching_level_sweeps_equal_row_form(shape, waves, monkeypatch):
    """The grid levels' pre-sweeps and last post-sweep in plane-marching form
    give the row form's bits (two coupled steps; levels of several sizes,
    ragged tiles, odd plane counts)."""
    out = []
    for zl in ("0", "1"):
        monkeypatch.setenv("HCA_MG_ZLEVELS", zl)
        monkeypatch.setenv("HCA_MG_ZL_WAVES", waves)
        sim, _, _ = make_pair(shape, "f32", seed=23, n_drugs=1, preconditioner=hca.HCA_PC_MG)
        sim.step(2)
        out.append((sim.states(), sim.field(hca.FIELD_O2), sim.field(hca.FIELD_O2_LO), sim.field(hca.FIELD_DRUG0),
                    sim.stats()))
        sim.close()
    a, b = out
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)
    assert a[4]["o2_iterations"] == b[4]["o2_iterations"]
    assert a[4]["drug_iterations"] == b[4]["drug_iterations"]
