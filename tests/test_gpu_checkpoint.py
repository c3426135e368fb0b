"""Checkpoint and resume (hca_save / hca_load): a run saved after some steps
and reloaded into a new handle continues bit for bit like the run that was
never interrupted — states, every field (with the FP32 defect-correction low
words), statistics and the step counter."""

import numpy as np
import pytest

from gpu_helpers import make_pair
from paper_2105_00448_gb300 import hca
from synth import make_maps

pytestmark = pytest.mark.gpu

CASES = [
    ("f64", dict(n_drugs=1)),
    ("f32", dict(n_drugs=2, preconditioner=hca.HCA_PC_MG, vegf=1, vessel_interval=2, V_high=5e-5,
                 beta_birth=0.5, drug_scheme=1, drug_substeps=2, pk_model=(0, 2, 0))),
    ("f32", dict(n_drugs=1, ca_mode=1, o2_nonlinear=1, picard_tol=1e-6)),
]


def _snapshot(sim, rep=0, vegf=False):
    bits = [hca.FIELD_O2, hca.FIELD_PHI, hca.FIELD_P53, hca.FIELD_VEGFC, hca.FIELD_PERF]
    bits += [hca.FIELD_DRUG[d] for d in range(sim.cfgs[rep].n_drugs)]
    if vegf:
        bits.append(hca.FIELD_VEGF)
    return [sim.states(rep)] + [sim.field(b, rep) for b in bits]


@pytest.mark.parametrize("precision,params", CASES)
def test_resume_is_bit_identical(precision, params, tmp_path):
    shape = (20, 24, 36)
    ref, _, _ = make_pair(shape, precision, seed=91, **params)
    ref.step(3)
    path = str(tmp_path / "run.ckpt")
    ref.save(path)
    res = hca.Sim.load(path)
    assert res.stats()["step"] == 3
    ref.step(3)
    res.step(3)
    vegf = bool(params.get("vegf"))
    for a, b in zip(_snapshot(ref, vegf=vegf), _snapshot(res, vegf=vegf)):
        assert np.array_equal(a, b)
    sa, sb = ref.stats(), res.stats()
    for k in ("step", "o2_iterations", "drug_iterations", "committed", "kills", "divisions", "counts",
              "vessel_births", "vessel_deaths"):
        assert sa[k] == sb[k], k
    ref.close()
    res.close()


def test_resume_batch(tmp_path):
    cfgs, maps = [], []
    for r, n in enumerate((16, 22)):
        m = make_maps(n, n, n, corr_len=3.0, seed=95 + r)
        maps.append((m.p_cell, m.perf, m.p_vessel))
        cfgs.append(hca.make_config(n, n, n, precision="f32", seed=95 + r, n_drugs=1,
                                    preconditioner=hca.HCA_PC_MG))
    ref = hca.Sim(cfgs, maps, batch=True)
    ref.step(2)
    path = str(tmp_path / "batch.ckpt")
    ref.save(path)
    res = hca.Sim.load(path)
    ref.step(2)
    res.step(2)
    for r in range(2):
        for a, b in zip(_snapshot(ref, r), _snapshot(res, r)):
            assert np.array_equal(a, b)
    ref.close()
    res.close()
