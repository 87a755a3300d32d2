"""Persistent contour sweeps over several replicas and row widths (Eq. 16-17), against the FP64
oracle: every row width the sweep supports (32, 48 and 64 sites: two rows per warp; 96 and 128
sites: one), a batch of mixed widths, chain lengths and species counts in shared launches,
bit-identity of a replica in the batch with its solo run, a race check, and the timeout of one
brick inside a batch, for bricks of 16 planes (one CTA per SM) and of 8 (two CTAs per SM).
Tolerance: FP32 <= 1e-5 relative to the field's largest magnitude.
"""
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


def t2n(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def melt(grid, N, nA, chiN=12.0, **kw):
    c = inputs.melt(grid, N, 0.5, chiN, **kw)
    c["nA"] = nA
    return c


def solution(grid, N, nA, phi_p=0.3, **kw):
    c = inputs.solution(grid, N, 0.3, phi_p, 20.0, 24.0, 3.0, **kw)
    c["nA"] = nA
    return c


def ncomp_shape(cfg):
    nx, ny, nz = cfg["grid"]
    return (cfg.get("ns", 2), nz, ny, nx)


@pytest.mark.parametrize("cfg", [melt((32, 16, 32), 7, 3), melt((48, 24, 16), 9, 4), solution((48, 8, 32), 6, 2),
                                 melt((48, 32, 16), 6, 2), melt((64, 16, 16), 5, 2), solution((64, 32, 16), 5, 2),
                                 melt((64, 8, 32), 6, 4), melt((96, 8, 32), 8, 5), solution((96, 16, 16), 7, 3)],
                         ids=lambda c: "x".join(map(str, c["grid"])) + f"_ns{c['ns']}")
@pytest.mark.parametrize("depth", [16, 8])
def test_persistent_row_widths_fp32_within_1e5(cfg, depth):
    """One replica per width: the two-rows-per-warp layouts (32, 48, 64), three sites per lane
    (48, 96) with the scalar tail of the packed pair arithmetic, and bricks of 16 rows (narrow
    rows with ny a multiple of 16) and of 8; bricks of 16 planes (one CTA per SM) and of 8 (two)."""
    if cfg["grid"][2] % depth:
        pytest.skip("brick depth does not divide nz")
    U = inputs.random_field(ncomp_shape(cfg), seed=21, scale=0.5)
    ref, _, _ = oracle.densities(cfg, U)
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set_tuning(depth, 0)
    assert ctx.diagnostics()["kfuse"] == 0
    for _ in range(2):      # the brick step counters carry over between launches
        got = t2n(ctx.densities(torch.from_numpy(U)))
        ctx.status()
        assert rel(got, ref) < 1e-5


BATCH = [melt((48, 16, 32), 8, 3), melt((64, 8, 16), 6, 2), melt((96, 16, 16), 9, 4), melt((48, 8, 16), 5, 4),
         solution((64, 16, 32), 7, 3), melt((32, 8, 16), 4, 1), melt((128, 8, 32), 6, 3)]


def _batch_U(cfgs, seed):
    return [inputs.random_field(ncomp_shape(c), seed=seed + r, scale=0.5) for r, c in enumerate(cfgs)]


def _split(flat, cfgs):
    out, o = [], 0
    for c in cfgs:
        n = int(np.prod(ncomp_shape(c)))
        out.append(flat[o:o + n].reshape(ncomp_shape(c)))
        o += n
    return out


@pytest.mark.parametrize("depth", [16, 8])
def test_persistent_batch_of_mixed_widths_matches_oracle_and_solo_runs(depth):
    """Seven replicas (widths 32 to 128, chain lengths 4 to 9, melts and a solution) in the
    persistent launches of one context: each against the oracle, and bit-identical to the same
    replica's own persistent sweep (a brick's arithmetic does not depend on the launch it is in)."""
    Us = _batch_U(BATCH, 30)
    ctx = dscf.Context(BATCH, dscf.FP32)
    ctx.set_tuning(depth, 0)
    assert ctx.diagnostics()["kfuse"] == 0
    flat = torch.cat([torch.from_numpy(U).float().reshape(-1) for U in Us])
    got = _split(ctx.densities(flat).cpu(), BATCH)
    ctx.status()
    for r, (cfg, U) in enumerate(zip(BATCH, Us)):
        ref, _, _ = oracle.densities(cfg, U)
        assert rel(got[r].numpy().astype(np.float64), ref) < 1e-5, r
        solo = dscf.Context(cfg, dscf.FP32)
        solo.set_tuning(depth, 0)
        one = solo.densities(torch.from_numpy(U)).cpu()
        solo.status()
        assert torch.equal(one, got[r]), r


@pytest.mark.parametrize("depth", [16, 8])
def test_persistent_batch_is_deterministic(depth):
    """Race check of the handshake with several replicas per launch: repeated density maps are
    bitwise equal."""
    Us = _batch_U(BATCH, 40)
    ctx = dscf.Context(BATCH, dscf.FP32)
    ctx.set_tuning(depth, 0)
    flat = torch.cat([torch.from_numpy(U).float().reshape(-1) for U in Us])
    first = ctx.densities(flat)
    for _ in range(10):
        assert torch.equal(ctx.densities(flat), first)
    ctx.status()


@pytest.mark.parametrize("depth", [16, 8])
def test_persistent_batch_timeout_is_reported_and_the_context_recovers(depth):
    """A lagging brick of one replica (host-side counter set far behind): its neighbours' bounded
    waits run out, the abort flag releases every CTA of every launch, the host reads
    DSCF_ERR_TIMEOUT, and the context computes the same densities again afterwards."""
    import time
    Us = _batch_U(BATCH, 50)
    ctx = dscf.Context(BATCH, dscf.FP32)
    ctx.set_tuning(depth, 0)
    flat = torch.cat([torch.from_numpy(U).float().reshape(-1) for U in Us])
    good = ctx.densities(flat)
    ctx.status()
    ctx.set_wait_limit(2000)
    ctx.inject_lag(0)   # brick 0 of the first replica, whose other brick then waits for it
    t0 = time.perf_counter()
    ctx.densities(flat)
    with pytest.raises(dscf.DSCFError) as err:
        ctx.status()
    assert err.value.code == -4
    assert time.perf_counter() - t0 < 30.0
    ctx.status()
    again = ctx.densities(flat)
    ctx.status()
    assert torch.equal(again, good)


@pytest.mark.parametrize("depth", [16, 8])
def test_persistent_batch_step_matches_multi_launch(depth):
    """A whole time step (inversion, LB, convection-diffusion) of a mixed batch with persistent
    sweeps against the single-step contour kernels."""
    cfgs = [melt((48, 16, 16), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4, seed=3),
            melt((96, 8, 16), 8, 3, hydro=1, ncg_iters=2, cn_sweeps=4, seed=4)]
    phis = [inputs.initial_fields(c) for c in cfgs]
    outs = []
    for kfuse, zc in ((1, 8), (0, depth)):
        ctx = dscf.Context(cfgs, dscf.FP32)
        ctx.set_tuning(zc, kfuse)
        ctx.set(dscf.PHI, torch.cat([torch.from_numpy(p).reshape(-1) for p in phis]).cuda())
        ctx.step(3)
        ctx.status()
        outs.append(t2n(ctx.get(dscf.PHI)))
    assert rel(outs[1], outs[0]) < 1e-5
