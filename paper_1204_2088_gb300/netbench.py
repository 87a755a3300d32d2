"""Timing of the predictor network's forward pass on one GPU.

    python -m paper_1204_2088_gb300.netbench [--grid 128 128 128] [--reps 10]

Prints, for the tcgen05 path (where the grid allows it) and the mma.sync path, the mean time of
one forward pass (CUDA events, after a warm-up pass) and the rate in TFLOP/s counted on the
padded channels (2 x 125 x (16 x 32 + 32 x 32 + 32 x 16) FLOP per site).  One further forward
pass on the default path is bracketed by cudaProfilerStart/Stop, so a profiler started with
profiling from start off captures exactly its kernels.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import dscf


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, nargs=3, default=[128, 128, 128])
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args()
    nx, ny, nz = a.grid
    net = dscf.Net((nx, ny, nz), 1, seed=1)
    g = torch.Generator(device="cuda").manual_seed(1)
    U = (torch.randn(1, 2, nz, ny, nx, device="cuda", generator=g) * 0.1).float()
    phibar = [0.5, 0.5]
    flop = 2.0 * nx * ny * nz * 125 * (16 * 32 + 32 * 32 + 32 * 16)
    out = {"grid": [nx, ny, nz]}
    for path in (0, 1):
        net.set_tensor_path(path)
        net.forward(U, phibar)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            net.forward(U, phibar)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        name = "tcgen05" if net.tensor_path() == 2 else "mma.sync"
        out[name] = {"ms": ms, "tflops_padded": flop / ms / 1e9}
    net.set_tensor_path(0)
    net.status()
    torch.cuda.profiler.start()
    net.forward(U, phibar)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    net.status()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
