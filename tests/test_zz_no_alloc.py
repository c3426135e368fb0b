"""hca_o2_residual_noalloc: the allocation-free oxygen residual check.

Callers that may not allocate device memory (inside another framework's
memory pool, or in a real-time loop that forbids cudaMalloc) cannot create a
handle just to check a field; this entry point takes their device arrays and
uses a fixed scratch array inside the library.  The test compares it with the
relative residual the existing handle path reports for the same oxygen solve
(hca_stage + hca_get_stats), on two calls in a row, at the 1e-12 tolerance
(relative to the size of the operator's terms) used for operator parity.
This file is collected last on purpose.
"""

import numpy as np
import pytest

from gpu_helpers import make_pair, random_states
from oracle import params as Pm
from paper_2105_00448_gb300 import hca

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(9, 17, 30), (24, 40, 64)])
def test_noalloc_residual_matches_handle_solve(shape):
    import torch

    rng = np.random.default_rng(5)
    sim, cfg, _ = make_pair(shape, "f64", seed=3, n_drugs=0, rtol_o2=1e-10, picard_maxit=1)
    st = random_states(shape, rng)
    st.reshape(-1)[0] = Pm.VESSEL
    K_prev = rng.uniform(0.0, 20.0, shape)
    sim.set_states(st)
    sim.set_field(hca.FIELD_O2, K_prev)
    sim.stage(hca.STAGE_O2)
    K = sim.field(hca.FIELD_O2)
    rel_handle = sim.stats()["o2_rel_residual"]
    sim.close()
    assert 0.0 < rel_handle <= 1e-10

    dev = torch.device("cuda", 0)
    st_d = torch.from_numpy(st.reshape(-1).copy()).to(dev)
    Kp_d = torch.from_numpy(K_prev.reshape(-1).copy()).to(dev)
    K_d = torch.from_numpy(K.reshape(-1).copy()).to(dev)
    nz, ny, nx = shape
    c = hca.make_config(nx, ny, nz)
    first = hca.hca_o2_residual_noalloc(c, st_d, Kp_d, K_d)
    second = hca.hca_o2_residual_noalloc(c, st_d, Kp_d, K_d)
    assert first == second
    assert abs(first - rel_handle) <= 1e-12
    # the starting field is far from the solution: a large residual, same on both calls
    rel0 = hca.hca_o2_residual_noalloc(c, st_d, Kp_d, Kp_d)
    assert rel0 > 1e-3 and rel0 == hca.hca_o2_residual_noalloc(c, st_d, Kp_d, Kp_d)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch

    dev = torch.device("cuda", 0)
    c = hca.make_config(4, 300, 300)          # 90000 rows > 65536
    st = torch.zeros(4 * 300 * 300, dtype=torch.uint8, device=dev)
    K = torch.zeros(4 * 300 * 300, dtype=torch.float64, device=dev)
    with pytest.raises(hca.HcaError) as e:
        hca.hca_o2_residual_noalloc(c, st, K, K)
    assert e.value.status == hca.HCA_ERR_ARG
