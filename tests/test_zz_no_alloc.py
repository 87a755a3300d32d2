"""The allocation-free density map (dscf_densities_static), called through the C ABI.

It serves callers that cannot allocate device memory; it must give the same densities as the
context-based dscf_densities (and as the FP64 oracle) on consecutive calls that reuse its fixed
scratch array, leave the caller's current device alone, and refuse problems larger than that
array.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
from paper_1204_2088_gb300 import build, dscf, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dscf.load()


def cfg_of(grid, N, nA, ns=2):
    if ns == 2:
        c = inputs.melt(grid, N, 0.5, 14.0)
    else:
        c = inputs.solution(grid, N, 0.3, 0.35, 20.0, 24.0, 3.0)
    c["nA"] = nA
    return c


@pytest.mark.parametrize("precision,tol", [(dscf.FP64, 1e-12), (dscf.FP32, 1e-5)])
def test_static_matches_context_entry_point_on_consecutive_calls(precision, tol):
    dtype = torch.float64 if precision == dscf.FP64 else torch.float32
    # two different problems in a row: the second reuses scratch the first left behind
    for cfg, seed in [(cfg_of((40, 20, 36), 8, 3), 1), (cfg_of((33, 17, 9), 7, 4, ns=3), 2),
                      (cfg_of((40, 20, 36), 8, 3), 3)]:
        nx, ny, nz = cfg["grid"]
        shape = (cfg["ns"], nz, ny, nx)
        U = torch.from_numpy(inputs.random_field(shape, seed=seed, scale=0.5)).to("cuda", dtype)
        out = torch.empty(shape, dtype=dtype, device="cuda")
        dev_before = torch.cuda.current_device()
        dscf.densities_static(cfg, U, out, precision)
        assert torch.cuda.current_device() == dev_before
        ref = dscf.Context(cfg, precision).densities(U)
        torch.cuda.synchronize()
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.abs(a - b).max() <= tol * np.abs(b).max()
        # and against the FP64 oracle on the same (rounded) potentials
        o = oracle.densities(cfg, U.double().cpu().numpy())[0]
        assert np.abs(a - o).max() <= tol * np.abs(o).max()


def test_static_rejects_problems_beyond_its_scratch():
    cfg = cfg_of((128, 128, 128), 64, 19)
    U = torch.zeros((2, 128, 128, 128), dtype=torch.float32, device="cuda")
    out = torch.full_like(U, -1.0)
    with pytest.raises(dscf.DSCFError) as e:
        dscf.densities_static(cfg, U, out, dscf.FP32)
    assert e.value.code == -3 and "DSCF_STATIC_SCRATCH_BYTES" in str(e.value)
    torch.cuda.synchronize()
    assert float(out.min()) == -1.0 and float(out.max()) == -1.0   # nothing was launched
