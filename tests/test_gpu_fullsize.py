"""Element-wise parity with the FP64 oracle at the size and in the launch configuration the
benchmark times, and over a long FP32 trajectory.

  - One coupled step of the 128^3 melt (N = 64, nA = 19, chi N = 25), FP32, in the tuning the
    autotuner picks for the benchmark (persistent contour sweeps: 128 bricks, one per SM), from a
    random state: every output field against the oracle's step from the same state.
  - One coupled step of the 48 mixed replicas (24 x 48^3, 16 x 64^3, 8 x 96^3) in the tuning the
    autotuner picks (persistent sweeps over the batch), three sampled replicas against the oracle.
  - 1000 FP32 steps of the 32^3 melt of the plain-method workload (N = 32, f = 0.5) at chi N = 8,
    below the spinodal, where rounding differences are damped instead of amplified: the
    compositions stay within 1e-5 of the FP64 oracle's trajectory (relative to their largest
    magnitude), and the composition fluctuations are tracked, not just their decay.  The time
    step is 0.1 tau: at 0.2 tau the explicit force/advection coupling of this configuration has a
    growing velocity mode (the oracle's own run reaches non-finite values after about 540 steps).
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


def test_bench_configuration_one_step_fp32_matches_oracle():
    cfg = inputs.workload("melt128")
    nx, ny, nz = cfg["grid"]
    shp = (2, nz, ny, nx)
    phi = inputs.initial_fields(dict(cfg, noise=0.04, seed=61))
    U = inputs.random_field(shp, seed=62, scale=0.2)
    _, w, _, _ = oracle.lb_basis()
    dn = 1e-3 * inputs.random_field((19, nz, ny, nx), seed=63) * w[:, None, None, None]
    # the FP32 context starts from the FP32-rounded state; the oracle from the same values
    phi32, U32, dn32 = (a.astype(np.float32).astype(np.float64) for a in (phi, U, dn))
    ctx = dscf.Context(cfg, dscf.FP32)
    d0 = ctx.diagnostics()
    assert d0["kfuse"] == 0, "the benchmark configuration runs the persistent sweeps"
    ctx.set(dscf.PHI, torch.from_numpy(phi32).float().cuda())
    ctx.set(dscf.U, torch.from_numpy(U32).float().cuda())
    ctx.set(dscf.POP, torch.from_numpy(dn32).float().cuda())
    ctx.step(1)
    ctx.status()
    got = {k: t2n(ctx.get(f)) for k, f in (("phi", dscf.PHI), ("U", dscf.U), ("mu", dscf.MU),
                                          ("ulat", dscf.VEL), ("pop", dscf.POP), ("phim", dscf.PHIM))}
    ctx.close()
    pop = dn32 + w[:, None, None, None]
    st = oracle.step(cfg, phi32, U32, pop, phi32.reshape(2, -1).sum(1))
    st["pop"] = st["pop"] - w[:, None, None, None]
    for k in ("phi", "U", "mu", "phim"):
        assert rel(got[k], st[k]) < 1e-5, (k, rel(got[k], st[k]))
    assert rel(got["ulat"], st["ulat"]) < 1e-4, rel(got["ulat"], st["ulat"])
    # population deviations (about 1e-3 w_i) carry the FP32 rounding of the full populations
    assert rel(got["pop"], st["pop"]) < 1e-4, rel(got["pop"], st["pop"])


def test_batch48_configuration_one_step_fp32_matches_oracle_on_sampled_replicas():
    """The 48 mixed replicas in the configuration the benchmark times (the autotuner's choice:
    persistent sweeps over the batch, mixed-width launches), one coupled step from a random state;
    three replicas, one of each size and chain length (48^3 N = 32, 64^3 N = 48, 96^3 N = 64),
    against the oracle's step of that replica alone."""
    cfgs = inputs.batch48()
    _, w, _, _ = oracle.lb_basis()
    states = []
    for r, c in enumerate(cfgs):
        nx, ny, nz = c["grid"]
        phi = inputs.initial_fields(dict(c, noise=0.04, seed=300 + r))
        U = inputs.random_field((2, nz, ny, nx), seed=400 + r, scale=0.2)
        dn = 1e-3 * inputs.random_field((19, nz, ny, nx), seed=500 + r) * w[:, None, None, None]
        states.append(tuple(a.astype(np.float32).astype(np.float64) for a in (phi, U, dn)))
    ctx = dscf.Context(cfgs, dscf.FP32)
    assert ctx.diagnostics()["kfuse"] == 0, "the benchmark configuration runs the persistent sweeps"
    for k, f in ((0, dscf.PHI), (1, dscf.U), (2, dscf.POP)):
        ctx.set(f, torch.cat([torch.from_numpy(st[k]).float().reshape(-1) for st in states]).cuda())
    ctx.step(1)
    ctx.status()
    got = {k: t2n(ctx.get(f)) for k, f in (("phi", dscf.PHI), ("U", dscf.U), ("mu", dscf.MU))}
    ctx.close()
    offs = np.cumsum([0] + [2 * int(np.prod(c["grid"])) for c in cfgs])
    for r in (0, 25, 41):
        c = cfgs[r]
        nx, ny, nz = c["grid"]
        phi32, U32, dn32 = states[r]
        st = oracle.step(c, phi32, U32, dn32 + w[:, None, None, None], phi32.reshape(2, -1).sum(1))
        for k in ("phi", "U", "mu"):
            mine = got[k][offs[r]:offs[r + 1]].reshape(2, nz, ny, nx)
            assert rel(mine, st[k]) < 1e-5, (r, k, rel(mine, st[k]))


def test_fp32_trajectory_of_1000_steps_stays_within_1e5_of_the_oracle():
    cfg = inputs.melt((32, 32, 32), 32, 0.5, 8.0, 1.0, 1.0, 0.01, 1, dt=0.1, name="melt32-chiN8")
    phi0 = inputs.initial_fields(cfg)
    phi32 = phi0.astype(np.float32).astype(np.float64)
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set(dscf.PHI, torch.from_numpy(phi32).float().cuda())
    _, w, _, _ = oracle.lb_basis()
    pop = np.broadcast_to(w[:, None, None, None], (19, 32, 32, 32)).copy()
    phi, U = phi32.copy(), np.zeros_like(phi32)
    m0 = phi32.reshape(2, -1).sum(1)
    worst, worst_dev = 0.0, 0.0
    for block in range(10):
        ctx.step(100)
        ctx.status()
        for _ in range(100):
            st = oracle.step(cfg, phi, U, pop, m0)
            phi, U, pop = st["phi"], st["U"], st["pop"]
        got = t2n(ctx.get(dscf.PHI))
        worst = max(worst, rel(got, phi))
        dev = phi - phi.reshape(2, -1).mean(1)[:, None, None, None]
        worst_dev = max(worst_dev, np.abs(got - phi).max() / np.abs(dev).max())
    print(f"1000 FP32 steps: max |phi - phi_oracle| / max|phi| = {worst:.3e}, "
          f"/ max|phi - <phi>| = {worst_dev:.3e}, fluctuation amplitude {np.abs(dev).max():.3e}")
    assert worst < 1e-5
    assert worst_dev < 1e-2
    assert np.abs(dev).max() > 1e-4          # the fluctuations have not all decayed
