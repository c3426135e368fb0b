"""Training helpers for the learned oxygen warm start (the network of hca.h's
"learned warm start" section).  Every step runs in libhca's kernels and the
training loop itself in one library call (hca_train_warmstart); this module
only draws the initial parameters and moves solver fields into device
tensors.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import hca

# conv layers in parameter order: (name, C_in, C_out)
CONVS = (("enc0", 16, 16), ("enc1", 16, 32), ("enc2", 32, 64), ("enc3", 64, 64),
         ("dec2", 64, 64), ("dec1", 64, 32), ("dec0", 32, 16))


def param_slices():
    """name -> (offset, shape) in the flat FP32 parameter array."""
    out, o = {}, 0
    for name, ci, co in CONVS:
        out[name + ".w"] = (o, (27, co, ci))
        o += 27 * co * ci
        out[name + ".b"] = (o, (co,))
        o += co
    out["head.w"] = (o, (16,))
    o += 16
    out["head.b"] = (o, (1,))
    o += 1
    out["_total"] = (o, ())
    return out


def init_params(seed: int) -> np.ndarray:
    """He-normal conv weights, zero biases, head weights ~ N(0, 1/16) scaled
    down so that the initial guess stays close to K_prev."""
    rng = np.random.default_rng(seed)
    sl = param_slices()
    flat = np.zeros(sl["_total"][0], dtype=np.float32)
    for name, ci, co in CONVS:
        o, shp = sl[name + ".w"]
        flat[o:o + int(np.prod(shp))] = (rng.standard_normal(int(np.prod(shp))) * np.sqrt(2.0 / (27 * ci)))
    o, _ = sl["head.w"]
    flat[o:o + 16] = rng.standard_normal(16) * 0.25 * 0.01
    return flat


@dataclass
class Sample:
    """One oxygen solve: the lattice it saw, K before and after (device tensors)."""
    state: object
    perf: object
    K_prev: object
    K_new: object


def collect_samples(sim: "hca.Sim", n_steps: int, device) -> List[Sample]:
    """Run n_steps full steps of a single-replicate simulation, recording each
    oxygen solve's input and solution as float32 device tensors."""
    import torch

    out = []
    perf = torch.from_numpy(sim.field(hca.FIELD_PERF).astype(np.float32).reshape(-1)).to(device)
    rest = hca.STAGE_DRUGS | hca.STAGE_ODE | hca.STAGE_CA | hca.STAGE_ADVANCE
    for _ in range(n_steps):
        st = torch.from_numpy(sim.states().reshape(-1).copy()).to(device)
        Kp = torch.from_numpy(sim.field(hca.FIELD_O2).astype(np.float32).reshape(-1)).to(device)
        sim.stage(hca.STAGE_O2)
        Kn = torch.from_numpy(sim.field(hca.FIELD_O2).astype(np.float32).reshape(-1)).to(device)
        sim.stage(rest)
        out.append(Sample(st, perf, Kp, Kn))
    return out


def train(net: "hca.Net", cfg: "hca.hca_config", samples: Sequence[Sample], iters: int, lr: float,
          seed: int = 0, lr_final: float = None, device=None, w_mse: float = 1.0, w_res: float = 0.0) -> np.ndarray:
    """iters Adam steps, each on one sample drawn (seeded) from samples; the
    learning rate decays geometrically to lr_final.  Returns the per-step
    losses (read back once at the end).

    The MSE term alone is the default: measured on held-out solves it cuts
    the oxygen CG iterations, while the residual term alone shrinks ||r0||
    far more but leaves smooth errors that CG removes slowly (more
    iterations)."""
    import torch

    dev = device if device is not None else samples[0].state.device
    losses = torch.zeros(max(1, iters), dtype=torch.float32, device=dev)
    lr_final = lr if lr_final is None else lr_final
    # one library call: the seeded sample order and the learning-rate
    # schedule run on the host side of libhca, every step in its kernels
    hca.hca_train_warmstart(net.handle, cfg, [s.state for s in samples], [s.perf for s in samples],
                            [s.K_prev for s in samples], [s.K_new for s in samples], iters, lr, lr_final,
                            seed=seed, w_mse=w_mse, w_res=w_res, losses=losses)
    hca.hca_net_sync(net.handle)
    return losses.cpu().numpy()[:iters]
