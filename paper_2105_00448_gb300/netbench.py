"""Time the warm-start network's kernels on one lattice (random inputs).

    python -m paper_2105_00448_gb300.netbench [--edge 128] [--reps 10]

Prints one JSON line: forward and forward+backward milliseconds (CUDA events
on the network's stream, after two warm-up passes) and the achieved
TFLOP/s of the convolutions (2 * 27 * C_in * C_out per output site; the
weight gradient and the input gradient each cost as much as the forward).
"""

from __future__ import annotations

import argparse
import json

import numpy as np

from . import hca, warmstart

# (C_in, C_out, level) of the seven 3x3x3 convolutions; the input gradient of
# enc0 is not computed
_CONVS = ((16, 16, 0), (16, 32, 1), (32, 64, 2), (64, 64, 3), (64, 64, 2), (64, 32, 1), (32, 16, 0))


def conv_flops(D: int, H: int, W: int):
    n0 = D * H * W
    fwd = sum(2 * 27 * ci * co * n0 / 8 ** lvl for ci, co, lvl in _CONVS)
    dgrad = fwd - 2 * 27 * 16 * 16 * n0
    return fwd, fwd + fwd + dgrad


def main(argv=None) -> int:
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--edge", type=int, default=128)
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    n = a.edge
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    net = hca.Net(n, n, n, trainable=True, stream=stream.cuda_stream)
    net.set_params(warmstart.init_params(0))
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.standard_normal(n ** 3 * 16).astype(np.float32)).to(dev).to(torch.bfloat16)
    tgt = torch.from_numpy(rng.standard_normal(n ** 3).astype(np.float32)).to(dev)
    out = torch.empty(n ** 3, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def timed(fn):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.reps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / a.reps

    fwd_ms = timed(lambda: hca.hca_net_forward_x(net.handle, x, out))
    bwd_ms = timed(lambda: hca.hca_net_gradients_x(net.handle, x, tgt, None, None))
    net.close()
    ff, fb = conv_flops(n, n, n)
    print(json.dumps({"lattice": [n] * 3, "forward_ms": fwd_ms, "forward_tflops": ff / fwd_ms / 1e9,
                      "fwd_bwd_ms": bwd_ms, "fwd_bwd_tflops": fb / bwd_ms / 1e9, "reps": a.reps}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
