"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 form <= 1e-10 relative to the field's largest magnitude, per step from an
identical state; FP32 form <= 1e-5 relative; batched replicas bit-identical to solo runs.
Full-size (128^3, N = 64) runs, too large for the oracle, are checked on properties that
hold at any size and on closed forms.
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


DENSITY_CASES = [
    melt((8, 8, 8), 4, 2),
    melt((32, 12, 10), 6, 3),          # whole-row layout, 1 site per lane
    melt((64, 9, 7), 7, 2),            # whole-row layout, 2 sites per lane, ragged y
    solution((128, 3, 5), 5, 2),       # whole-row layout, 4 sites per lane, solvent
    melt((40, 20, 36), 8, 3),          # several tiles in x, y and z, ragged in each
    solution((33, 17, 9), 7, 4),       # solvent, odd sizes
    melt((1, 3, 70), 5, 2),            # degenerate x, z chunking with a ragged tail
    melt((256, 9, 5), 6, 2),           # whole rows of 256 sites (8 per lane, kernels of their own), ragged y
]


def ncomp_shape(cfg):
    nx, ny, nz = cfg["grid"]
    return (cfg.get("ns", 2), nz, ny, nx)


@pytest.mark.parametrize("cfg", DENSITY_CASES, ids=lambda c: "x".join(map(str, c["grid"])) + f"_N{c['N']}_ns{c['ns']}")
def test_densities_fp64_match_oracle(cfg):
    U = inputs.random_field(ncomp_shape(cfg), seed=7, scale=0.5)
    ref, _, _ = oracle.densities(cfg, U)
    ctx = dscf.Context(cfg, dscf.FP64)
    got = t2n(ctx.densities(torch.from_numpy(U)))
    ctx.status()
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("cfg", DENSITY_CASES, ids=lambda c: "x".join(map(str, c["grid"])) + f"_N{c['N']}_ns{c['ns']}")
def test_densities_fp32_within_1e5(cfg):
    U = inputs.random_field(ncomp_shape(cfg), seed=8, scale=0.5)
    ref, _, _ = oracle.densities(cfg, U)
    ctx = dscf.Context(cfg, dscf.FP32)
    got = t2n(ctx.densities(torch.from_numpy(U)))
    assert rel(got, ref) < 1e-5


FUSED_CASES = [
    (melt((32, 12, 10), 9, 4), 5),
    (melt((64, 9, 21), 11, 3), 8),
    (solution((128, 10, 6), 7, 5), 4),
    (melt((256, 11, 9), 7, 3), 4),     # rows of 256 sites: at most two steps per launch
]


@pytest.mark.parametrize("kfuse", [1, 2, 3, 4])
@pytest.mark.parametrize("case", FUSED_CASES, ids=lambda c: "x".join(map(str, c[0]["grid"])) + f"_zc{c[1]}")
def test_fused_contour_groups_fp32_within_1e5(case, kfuse):
    """Every contour-fusion depth (including groups that straddle the A/B junction and short
    last groups) gives the oracle's densities within the FP32 tolerance."""
    cfg, zc = case
    U = inputs.random_field(ncomp_shape(cfg), seed=9, scale=0.5)
    ref, _, _ = oracle.densities(cfg, U)
    ctx = dscf.Context(cfg, dscf.FP32)
    if cfg["grid"][0] == 256 and kfuse > 2:
        with pytest.raises(dscf.DSCFError):
            ctx.set_tuning(zc, kfuse)
        return
    ctx.set_tuning(zc, kfuse)
    got = t2n(ctx.densities(torch.from_numpy(U)))
    assert ctx.diagnostics()["kfuse"] == kfuse
    assert rel(got, ref) < 1e-5


PERSISTENT_CASES = [melt((128, 16, 32), 7, 3), solution((128, 8, 24), 6, 4), melt((128, 24, 16), 12, 5)]


@pytest.mark.parametrize("depth", [8, 16])
@pytest.mark.parametrize("cfg", PERSISTENT_CASES, ids=lambda c: "x".join(map(str, c["grid"])) + f"_ns{c['ns']}")
def test_persistent_sweeps_fp32_within_1e5(cfg, depth):
    """One-launch-per-sweep contour kernel (bricks exchanging halos through L2) against the oracle,
    with bricks of 16 planes (one CTA per SM) and of 8 planes (two CTAs per SM)."""
    if cfg["grid"][2] % depth:
        pytest.skip("brick depth does not divide nz")
    U = inputs.random_field(ncomp_shape(cfg), seed=10, scale=0.5)
    ref, _, _ = oracle.densities(cfg, U)
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set_tuning(depth, 0)
    assert ctx.diagnostics()["kfuse"] == 0
    for _ in range(2):      # twice: the brick step counters carry over between launches
        got = t2n(ctx.densities(torch.from_numpy(U)))
        ctx.status()
        assert rel(got, ref) < 1e-5


@pytest.mark.parametrize("depth,case", [(8, 0), (16, 0), (16, 2)])
def test_persistent_sweeps_are_deterministic(depth, case):
    """Race check of the brick handshake (release store after the CTA barrier, acquire loads of
    the neighbours' counters): the density map of the persistent sweep, repeated, is bitwise the
    same every time (a halo row read before its neighbour published it would perturb it); also
    with a single brick along z, its own z-neighbour."""
    cfg = PERSISTENT_CASES[case]
    U = torch.from_numpy(inputs.random_field(ncomp_shape(cfg), seed=13, scale=0.5))
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set_tuning(depth, 0)
    first = ctx.densities(U)
    for _ in range(20):
        assert torch.equal(ctx.densities(U), first)
    ctx.status()


@pytest.mark.parametrize("depth", [8, 16])
def test_persistent_sweep_timeout_is_reported_and_the_context_recovers(depth):
    """Failure detection without a GPU fault: one brick's step counter is set far behind (host
    side), so its neighbours wait for a value nobody publishes; their bounded waits run out, the
    abort flag releases every other CTA, the launch finishes and the host reads DSCF_ERR_TIMEOUT.
    The same context then computes correct densities again."""
    import time
    cfg = PERSISTENT_CASES[0]
    U = torch.from_numpy(inputs.random_field(ncomp_shape(cfg), seed=12, scale=0.5))
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set_tuning(depth, 0)
    good = ctx.densities(U)
    ctx.status()
    ctx.set_wait_limit(2000)
    ctx.inject_lag(0)
    t0 = time.perf_counter()
    ctx.densities(U)
    with pytest.raises(dscf.DSCFError) as err:
        ctx.status()
    assert err.value.code == -4
    assert time.perf_counter() - t0 < 30.0
    ctx.status()                    # re-armed by the call that reported the timeout
    again = ctx.densities(U)
    ctx.status()
    assert torch.equal(again, good)
    with pytest.raises(dscf.DSCFError):
        ctx.inject_lag(1000)
    with pytest.raises(dscf.DSCFError):
        ctx.set_wait_limit(0)


def test_persistent_step_matches_multi_launch():
    cfg = melt((128, 16, 16), 8, 3, hydro=1, ncg_iters=2, cn_sweeps=4)
    phi, U, dn = random_state(cfg, 91)
    outs = []
    for kfuse, zc in ((1, 8), (0, 8), (0, 16)):
        ctx = dscf.Context(cfg, dscf.FP32)
        ctx.set_tuning(zc, kfuse)
        ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
        ctx.set(dscf.U, torch.from_numpy(U).cuda())
        ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
        ctx.step(3)
        ctx.status()
        outs.append(t2n(ctx.get(dscf.PHI)))
    assert rel(outs[1], outs[0]) < 1e-5 and rel(outs[2], outs[0]) < 1e-5


def test_cached_tuning_reproduces_the_autotuned_context(tmp_path):
    cfg = melt((128, 16, 16), 8, 3, hydro=1, ncg_iters=2, cn_sweeps=4)
    phi, U, dn = random_state(cfg, 93)
    cache = tmp_path / "tuning.json"
    outs, tunings = [], []
    for _ in range(2):   # the first context runs the autotuner and writes the cache, the second reads it
        ctx = dscf.Context(cfg, dscf.FP32, tuning_cache=str(cache))
        d = ctx.diagnostics()
        tunings.append((d["zc"], d["kfuse"]))
        assert cache.exists()
        ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
        ctx.set(dscf.U, torch.from_numpy(U).cuda())
        ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
        ctx.step(2)
        ctx.status()
        outs.append(t2n(ctx.get(dscf.PHI)))
    assert tunings[0] == tunings[1]
    assert np.array_equal(outs[0], outs[1])
    with pytest.raises(dscf.DSCFError):
        dscf.Context(cfg, dscf.FP32, tuning=(4, 9))
    bad = melt((40, 16, 16), 8, 3, hydro=1)
    with pytest.raises(dscf.DSCFError):
        dscf.Context(bad, dscf.FP32, tuning=(8, 0))   # persistent sweeps need nx in {32, 48, 64, 96, 128}


def test_fused_step_fp32_matches_single_step():
    cfg = melt((32, 16, 24), 10, 4, hydro=1, ncg_iters=2, cn_sweeps=4)
    phi, U, dn = random_state(cfg, 81)
    outs = []
    for kfuse in (1, 3):
        ctx = dscf.Context(cfg, dscf.FP32)
        ctx.set_tuning(6, kfuse)
        ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
        ctx.set(dscf.U, torch.from_numpy(U).cuda())
        ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
        ctx.step(2)
        outs.append(t2n(ctx.get(dscf.PHI)))
    o = run_oracle(cfg, phi, U, dn, 2)
    assert rel(outs[1], outs[0]) < 1e-5
    assert rel(outs[1], o["phi"]) < 1e-5


def random_state(cfg, seed):
    shp = ncomp_shape(cfg)
    phi = inputs.initial_fields(dict(cfg, noise=0.04, seed=seed))
    U = inputs.random_field(shp, seed=seed + 1, scale=0.2)
    nx, ny, nz = cfg["grid"]
    _, w, _, _ = oracle.lb_basis()
    dn = 1e-3 * inputs.random_field((19, nz, ny, nx), seed=seed + 2) * w[:, None, None, None]
    return phi, U, dn


def run_gpu(cfg, prec, phi, U, dn, steps):
    ctx = dscf.Context(cfg, prec)
    ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
    ctx.set(dscf.U, torch.from_numpy(U).cuda())
    ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
    ctx.step(steps)
    ctx.status()
    out = {k: t2n(ctx.get(w)) for k, w in
           [("phi", dscf.PHI), ("U", dscf.U), ("mu", dscf.MU), ("ulat", dscf.VEL), ("pop", dscf.POP), ("phim", dscf.PHIM)]}
    out["diag"] = ctx.diagnostics()
    ctx.close()
    return out


def run_oracle(cfg, phi, U, dn, steps):
    _, w, _, _ = oracle.lb_basis()
    pop = dn + cfg.get("rho0", 1.0) * w[:, None, None, None]
    m0 = phi.reshape(phi.shape[0], -1).sum(1)
    st = None
    for _ in range(steps):
        st = oracle.step(cfg, phi, U, pop, m0)
        phi, U, pop = st["phi"], st["U"], st["pop"]
    st["pop"] = st["pop"] - cfg.get("rho0", 1.0) * w[:, None, None, None]
    return st


STEP_CASES = [
    melt((20, 12, 16), 6, 3, hydro=1, ncg_iters=3, cn_sweeps=4),
    melt((64, 10, 12), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4),
    melt((20, 12, 16), 6, 3, hydro=0, ncg_iters=3, cn_sweeps=4),
    solution((18, 10, 34), 5, 2, hydro=1, ncg_iters=2, cn_sweeps=6),
    melt((36, 9, 10), 8, 5, hydro=1, ncg_iters=4, cn_sweeps=8, dt=0.4, tau_s=0.7, tau_b=1.4),
]


@pytest.mark.parametrize("cfg", STEP_CASES, ids=lambda c: "x".join(map(str, c["grid"])) + f"_ns{c['ns']}_h{c['hydro']}")
def test_step_fp64_matches_oracle(cfg):
    phi, U, dn = random_state(cfg, 31)
    for steps in (1, 3):
        g = run_gpu(cfg, dscf.FP64, phi, U, dn, steps)
        o = run_oracle(cfg, phi, U, dn, steps)
        for k in ("phi", "U", "mu", "phim"):
            assert rel(g[k], o[k]) < 1e-10, (k, steps, rel(g[k], o[k]))
        if cfg["hydro"]:
            assert rel(g["ulat"], o["ulat"]) < 1e-10
            assert rel(g["pop"], o["pop"]) < 1e-10
        else:
            assert np.abs(g["ulat"]).max() == 0.0


def test_ncg_history_matches_oracle():
    cfg = STEP_CASES[0]
    phi, U, dn = random_state(cfg, 41)
    g = run_gpu(cfg, dscf.FP64, phi, U, dn, 1)
    o = run_oracle(cfg, phi, U, dn, 1)
    info = o["info"]
    assert abs(g["diag"]["gg_start"] - info[0]) < 1e-10 * info[0]
    assert abs(g["diag"]["gmax_end"] - info[-1]) < 1e-10 * max(info[-1], 1e-300) + 1e-16


def _stop_point(info, K, margin):
    """An iteration j and a tolerance that stops the inversion there with relative margin
    `margin` on both sides (residuals r_0..r_{j-1} above it, r_j below it)."""
    r = [info[1]] + [info[2 + 4 * k + 3] for k in range(K)]
    for j in (3, 2, 4, 1, 5):
        tol = (1.0 + margin) * r[j]
        if min(r[:j]) > (1.0 + margin) * tol:
            return j, tol
    raise AssertionError(f"no clean stop point in {r}")


def _iters_run(info, K, tol):
    r = [info[1]] + [info[2 + 4 * k + 3] for k in range(K)]
    k = next((k for k in range(K) if not r[k] >= tol), K)
    return k, min(abs(x / tol - 1.0) for x in r[:k + 1] if x != 0.0)


def test_residual_stop_fp64_matches_oracle():
    cfg = melt((20, 12, 16), 6, 3, hydro=1, ncg_iters=8, cn_sweeps=4)
    phi, U, dn = random_state(cfg, 61)
    j, tol = _stop_point(run_oracle(cfg, phi, U, dn, 1)["info"], 8, 0.01)
    for t in (tol, 10.0):   # a stop inside the inversion; a tolerance no residual reaches
        ctx = dscf.Context(cfg, dscf.FP64)
        ctx.set_inversion_tol(t)
        ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
        ctx.set(dscf.U, torch.from_numpy(U).cuda())
        ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
        ocfg = dict(cfg, ncg_tol=t)
        _, w, _, _ = oracle.lb_basis()
        oph, oU, opop = phi, U, dn + w[:, None, None, None]
        m0 = phi.reshape(phi.shape[0], -1).sum(1)
        for step in range(3):
            ctx.step(1)
            ctx.status()
            st = oracle.step(ocfg, oph, oU, opop, m0)
            oph, oU, opop = st["phi"], st["U"], st["pop"]
            k, gap = _iters_run(st["info"], 8, t)
            assert gap > 1e-6   # the FP64 decision cannot flip on rounding
            d = ctx.diagnostics()
            assert d["ncg_iters"] == k
            if step == 0:
                assert k == (j if t == tol else 0)
            for name, which, ref in (("phi", dscf.PHI, oph), ("U", dscf.U, oU), ("phim", dscf.PHIM, st["phim"]),
                                     ("mu", dscf.MU, st["mu"])):
                assert rel(t2n(ctx.get(which)), ref) < 1e-10, (t, step, name)
        ctx.close()


def test_residual_stop_with_persistent_and_multi_launch_sweeps():
    cfg = melt((128, 16, 16), 8, 3, hydro=1, ncg_iters=6, cn_sweeps=4)
    phi, U, dn = random_state(cfg, 63)
    j, tol = _stop_point(run_oracle(cfg, phi, U, dn, 1)["info"], 6, 0.05)
    o = run_oracle(dict(cfg, ncg_tol=tol), phi, U, dn, 1)
    for zc, kfuse in ((16, 0), (8, 1), (8, 4)):
        ctx = dscf.Context(cfg, dscf.FP32, tuning=(zc, kfuse))
        ctx.set_inversion_tol(tol)
        ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
        ctx.set(dscf.U, torch.from_numpy(U).cuda())
        ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
        ctx.step(1)
        ctx.status()
        assert ctx.diagnostics()["ncg_iters"] == j, (zc, kfuse)
        assert rel(t2n(ctx.get(dscf.PHI)), o["phi"]) < 1e-5
        assert rel(t2n(ctx.get(dscf.U)), o["U"]) < 1e-5
        ctx.close()
    with pytest.raises(dscf.DSCFError):
        ctx = dscf.Context(cfg, dscf.FP32)
        ctx.set_inversion_tol(-1.0)


ROW_CASES = [
    melt((128, 8, 6), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4),
    solution((128, 6, 4), 5, 2, hydro=1, ncg_iters=2, cn_sweeps=4),
    melt((64, 10, 12), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=6),
    melt((32, 12, 8), 6, 3, hydro=0, ncg_iters=2, cn_sweeps=6),
]


@pytest.mark.parametrize("cfg", ROW_CASES, ids=lambda c: "x".join(map(str, c["grid"])) + f"_ns{c['ns']}")
def test_step_fp32_row_kernels_within_tolerance(cfg):
    """FP32 step on grids whose x rows fill whole warps (nx = 128: chemical potentials one warp per
    row; nx dividing 128: Jacobi x neighbours by shuffles), melt and solution, two steps."""
    phi, U, dn = random_state(cfg, 57)
    g = run_gpu(cfg, dscf.FP32, phi, U, dn, 2)
    o = run_oracle(cfg, phi, U, dn, 2)
    for k in ("phi", "U", "mu", "phim"):
        assert rel(g[k], o[k]) < 1e-5, (k, rel(g[k], o[k]))


NOISE_CASES = [
    (melt((20, 12, 16), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4), dscf.FP64),
    (melt((20, 12, 16), 6, 3, hydro=0, ncg_iters=2, cn_sweeps=4), dscf.FP64),
    (solution((18, 10, 14), 5, 2, hydro=1, ncg_iters=2, cn_sweeps=4), dscf.FP64),
    (melt((128, 8, 6), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4), dscf.FP32),
    (solution((128, 6, 4), 5, 2, hydro=1, ncg_iters=2, cn_sweeps=4), dscf.FP32),
    (melt((20, 12, 16), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4), dscf.FP32),
]


@pytest.mark.parametrize("cfg,prec", NOISE_CASES,
                         ids=lambda v: "x".join(map(str, v["grid"])) + f"_ns{v['ns']}_h{v['hydro']}" if isinstance(v, dict) else ("fp64" if v == dscf.FP64 else "fp32"))
def test_thermal_noise_step_matches_oracle(cfg, prec):
    """Steps with thermal noise (Eq. 5 compositions, Eq. 13 LB modes, Omega = 100) against the
    oracle drawing the same Philox normals: FP64 within 1e-10, FP32 within 1e-5, three steps;
    the noise changes the result and keeps every species' mass."""
    seed, omega = 0x1234_5678_9ABC, 100.0
    phi, U, dn = random_state(cfg, 97)
    ctx = dscf.Context(cfg, prec)
    ctx.set_noise(omega, lb_noise=True, seed=seed)
    ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
    ctx.set(dscf.U, torch.from_numpy(U).cuda())
    ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
    _, w, _, _ = oracle.lb_basis()
    oph, oU, opop = phi, U, dn + w[:, None, None, None]
    m0 = phi.reshape(phi.shape[0], -1).sum(1)
    tol = 1e-10 if prec == dscf.FP64 else 1e-5
    for step in range(3):
        ctx.step(1)
        ctx.status()
        ocfg = dict(cfg, omega=omega, lb_noise=1, noise_seed=seed, noise_step=step)
        st = oracle.step(ocfg, oph, oU, opop, m0)
        oph, oU, opop = st["phi"], st["U"], st["pop"]
        assert rel(t2n(ctx.get(dscf.PHI)), oph) < tol, step
        assert rel(t2n(ctx.get(dscf.U)), oU) < tol, step
        if cfg["hydro"]:
            assert rel(t2n(ctx.get(dscf.POP)), opop - w[:, None, None, None]) < tol, step
    got = t2n(ctx.get(dscf.PHI))
    mtol = 1e-9 if prec == dscf.FP64 else 1e-6   # FP32 storage of the fields
    assert np.abs(got.reshape(phi.shape[0], -1).sum(1) - m0).max() < mtol * m0.max()
    quiet = run_oracle(cfg, phi, U, dn, 3)
    assert rel(got, quiet["phi"]) > 10 * tol   # the noise is there


def test_step_fp32_within_tolerance():
    cfg = STEP_CASES[0]
    phi, U, dn = random_state(cfg, 51)
    g = run_gpu(cfg, dscf.FP32, phi, U, dn, 1)
    o = run_oracle(cfg, phi, U, dn, 1)
    assert rel(g["phi"], o["phi"]) < 1e-5
    assert rel(g["mu"], o["mu"]) < 1e-5
    assert rel(g["pop"], o["pop"]) < 1e-4   # deviations of order 1e-5 stored in FP32


def test_batched_replicas_bit_identical_to_solo():
    cfgs = [melt((12, 10, 8), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4),
            melt((40, 9, 17), 9, 4, hydro=1, ncg_iters=2, cn_sweeps=4, tau_s=0.8),
            solution((10, 10, 10), 4, 2, hydro=1, ncg_iters=2, cn_sweeps=4)]
    states = [random_state(c, 60 + 3 * i) for i, c in enumerate(cfgs)]
    ctx = dscf.Context(cfgs, dscf.FP64)
    ctx.set(dscf.PHI, torch.from_numpy(np.concatenate([s[0].ravel() for s in states])).cuda())
    ctx.set(dscf.U, torch.from_numpy(np.concatenate([s[1].ravel() for s in states])).cuda())
    ctx.set(dscf.POP, torch.from_numpy(np.concatenate([s[2].ravel() for s in states])).cuda())
    ctx.step(2)
    ctx.status()
    phi_b = t2n(ctx.get(dscf.PHI))
    off = 0
    for c, (phi, U, dn) in zip(cfgs, states):
        solo = run_gpu(c, dscf.FP64, phi, U, dn, 2)
        n = phi.size
        assert np.array_equal(phi_b[off:off + n], solo["phi"].ravel())
        off += n


def test_large_batch_matches_solo_to_rounding():
    """A batch large enough to take a common flat chunk (here 2 x 48^3 + 32^3 sites) regroups
    the FP64 block partials, so it matches the solo runs to rounding rather than bit for bit."""
    cfgs = [melt((48, 48, 48), 6, 3, hydro=1, ncg_iters=2, cn_sweeps=4),
            melt((48, 48, 48), 8, 3, hydro=1, ncg_iters=2, cn_sweeps=4, tau_s=0.8),
            solution((32, 32, 32), 5, 2, hydro=1, ncg_iters=2, cn_sweeps=4)]
    states = [random_state(c, 70 + 3 * i) for i, c in enumerate(cfgs)]
    ctx = dscf.Context(cfgs, dscf.FP64)
    ctx.set(dscf.PHI, torch.from_numpy(np.concatenate([s[0].ravel() for s in states])).cuda())
    ctx.set(dscf.U, torch.from_numpy(np.concatenate([s[1].ravel() for s in states])).cuda())
    ctx.set(dscf.POP, torch.from_numpy(np.concatenate([s[2].ravel() for s in states])).cuda())
    ctx.step(2)
    ctx.status()
    phi_b, U_b = t2n(ctx.get(dscf.PHI)), t2n(ctx.get(dscf.U))
    off = 0
    for c, (phi, U, dn) in zip(cfgs, states):
        solo = run_gpu(c, dscf.FP64, phi, U, dn, 2)
        n = phi.size
        assert rel(phi_b[off:off + n], solo["phi"].ravel()) < 1e-12
        assert rel(U_b[off:off + n], solo["U"].ravel()) < 1e-10
        off += n


@pytest.mark.parametrize("cfg", [STEP_CASES[0], STEP_CASES[3]], ids=["melt", "solution"])
def test_observables_match_oracle(cfg):
    """Free energy (Eq. 1), order parameter (Fig. 1) and segregation (Fig. 3) of the GPU's own
    state after two steps against the oracle's functions of the same fields: FP64 to 1e-10, FP32
    to the FP32 bound."""
    phi, U, dn = random_state(cfg, 71)
    for prec, tol in ((dscf.FP64, 1e-10), (dscf.FP32, 2e-5)):
        ctx = dscf.Context(cfg, prec)
        ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
        ctx.set(dscf.U, torch.from_numpy(U).cuda())
        ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
        ctx.step(2)
        obs = ctx.observables()
        ctx.status()
        gphi, gU = t2n(ctx.get(dscf.PHI)), t2n(ctx.get(dscf.U))
        F = oracle.free_energy(cfg, gU, gphi)
        S = oracle.order_parameter(cfg, gphi)
        seg = oracle.segregation(cfg, gphi)
        # F is a difference of O(1) terms: compare on the scale of its largest term
        scale = max(abs(F), float(np.abs(gU * gphi).sum(0).mean()), 1.0)
        assert abs(obs["free_energy"] - F) < tol * scale, (prec, obs["free_energy"], F)
        assert abs(obs["order_parameter"] - S) < tol * S + 1e-12, (prec, obs["order_parameter"], S)
        assert abs(obs["segregation"] - seg) < tol * max(seg, 1e-3), (prec, obs["segregation"], seg)


def test_lb_step_alone_with_external_force():
    cfg = melt((14, 9, 11), 4, 2, tau_s=0.65, tau_b=1.7)
    _, w, _, _ = oracle.lb_basis()
    nx, ny, nz = cfg["grid"]
    dn = 2e-3 * inputs.random_field((19, nz, ny, nx), seed=71) * w[:, None, None, None]
    f = 1e-4 * inputs.random_field((3, nz, ny, nx), seed=72)
    ctx = dscf.Context(cfg, dscf.FP64)
    ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
    ctx.lb_step(torch.from_numpy(f).cuda(), 2)
    got = t2n(ctx.get(dscf.POP))
    n = dn + w[:, None, None, None]
    for _ in range(2):
        n, u = oracle.lb_step(cfg, n, f)
    assert rel(got, n - w[:, None, None, None]) < 1e-12
    assert rel(t2n(ctx.get(dscf.VEL)), u) < 1e-12


# ---------------------------------------------------------------------------------------------
# Full size, in the configuration the benchmark times (FP32, 128^3, N = 64, nA = 19)
# ---------------------------------------------------------------------------------------------
def full_cfg():
    return inputs.workload("melt128")


def test_full_size_homogeneous_field_closed_form():
    cfg = full_cfg()
    ctx = dscf.Context(cfg, dscf.FP32)
    nx, ny, nz = cfg["grid"]
    U = torch.empty((2, nz, ny, nx), dtype=torch.float32, device="cuda")
    U[0] = 0.03
    U[1] = -0.02
    phi = t2n(ctx.densities(U))
    f = cfg["nA"] / cfg["N"]
    assert np.abs(phi[0] - f).max() < 2e-6 and np.abs(phi[1] - (1 - f)).max() < 2e-6


def test_full_size_linear_response_closed_form():
    """A small plane-wave potential dU_I cos(k.r) gives dphi = -S(k) dU with the discrete Debye
    matrix S_IJ(k) = (phi_p/N) sum_{s in I, s' in J} sigma_hat(k)^|s-s'| (first order in dU)."""
    cfg = full_cfg()
    nx, ny, nz = cfg["grid"]
    k = (2 * np.pi * 3 / nx, 2 * np.pi * 1 / ny, 0.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wave = np.cos(k[0] * x + k[1] * y)
    dU = np.array([1e-3, -0.6e-3])
    U = (dU[:, None, None, None] * wave[None]).astype(np.float32)
    ctx = dscf.Context(cfg, dscf.FP32)
    phi = t2n(ctx.densities(torch.from_numpy(U)))
    N, nA = cfg["N"], cfg["nA"]
    al = cfg["a"] ** 2 / 6
    sh = np.prod([1 - 2 * al + 2 * al * np.cos(kk) for kk in k])
    types = np.array([0] * nA + [1] * (N - nA))
    S = np.zeros((2, 2))
    for s in range(N):
        np.add.at(S[types[s]], types, sh ** np.abs(s - np.arange(N)))
    S /= N
    expect = -S @ dU
    wv = wave.ravel()
    meas = np.array([((phi[I].ravel() - phi[I].mean()) * wv).sum() / (wv * wv).sum() for I in range(2)])
    assert np.abs(meas - expect).max() < 2e-3 * np.abs(expect).max()


def test_full_size_step_conserves_mass_and_stays_finite():
    cfg = full_cfg()
    phi0 = inputs.initial_fields(cfg)
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set(dscf.PHI, torch.from_numpy(phi0).float().cuda())
    ctx.step(3)
    ctx.status()
    d = ctx.diagnostics()
    phi = t2n(ctx.get(dscf.PHI))
    m0 = phi0.astype(np.float32).astype(np.float64).reshape(2, -1).sum(1)
    assert np.abs(phi.reshape(2, -1).sum(1) - m0).max() < 1e-6 * m0.max()
    assert abs(d["lb_mass"] - np.prod(cfg["grid"])) < 1e-6 * np.prod(cfg["grid"])
    # a 4-iteration Fletcher-Reeves inversion from a cold start at N = 64 is not converged
    # (the low-wavevector density response is ~N f times stiffer than the local one); its
    # residual stays bounded and finite
    assert np.isfinite(d["gmax_end"]) and d["gmax_end"] < 0.1
    assert np.isfinite(phi).all() and d["umax"] < 0.1


def test_error_codes():
    cfg = melt((8, 8, 8), 4, 2)
    ctx = dscf.Context(cfg, dscf.FP64)
    with pytest.raises(dscf.DSCFError) as e:
        ctx.set(dscf.MU, torch.zeros(ncomp_shape(cfg), dtype=torch.float64, device="cuda"))
    assert e.value.code == -1
    lib = dscf.load()
    import ctypes
    p = dscf.make_params(cfg)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    rc = lib.dscf_init(ctypes.byref(p), 1, 0, ctypes.c_void_p(ws.data_ptr()), 1024, None, ctypes.byref(h))
    assert rc == -3 and not h.value


@pytest.mark.parametrize("tol", [0.0, 1e-7], ids=["fixed_count", "residual_stop"])
def test_extrapolated_warm_start_fp64_matches_oracle(tol):
    """The inversion started from 2 U^{n-1} - U^{n-2} (dscf_set_warm_start(1)), against the oracle
    step by step: the history starts after dscf_set_fields (the first two steps start from
    U^{n-1}), the starting densities are evaluated at the extrapolated potentials."""
    cfg = dict(STEP_CASES[0], ncg_iters=3 if tol == 0.0 else 12)
    phi, U, dn = random_state(cfg, 71)
    ctx = dscf.Context(cfg, dscf.FP64)
    ctx.set(dscf.PHI, torch.from_numpy(phi).cuda())
    ctx.set(dscf.U, torch.from_numpy(U).cuda())
    ctx.set(dscf.POP, torch.from_numpy(dn).cuda())
    ctx.set_warm_start(1)
    if tol > 0:
        ctx.set_inversion_tol(tol)
    _, w, _, _ = oracle.lb_basis()
    pop = dn + w[:, None, None, None]
    m0 = phi.reshape(2, -1).sum(1)
    ocfg = dict(cfg, warm_extrap=1, ncg_tol=tol)
    Up = None
    for k in range(5):
        ctx.step(1)
        ctx.status()
        st = oracle.step(ocfg, phi, U, pop, m0, Uprev=Up if k >= 2 else None)
        phi, U, pop, Up = st["phi"], st["U"], st["pop"], st["Uprev"]
        for name, which, ref in (("phi", dscf.PHI, phi), ("U", dscf.U, U), ("mu", dscf.MU, st["mu"]),
                                 ("phim", dscf.PHIM, st["phim"])):
            assert rel(t2n(ctx.get(which)), ref) < 1e-10, (k, name)
        if tol > 0:
            its = sum(1 for j in range(12) if st["info"][2 + 4 * j + 3] != 0.0)
            assert ctx.diagnostics()["ncg_iters"] == its, k
    ctx.close()


def test_host_buffers_round_trip_and_pinned_upload_is_ordered():
    """Fields through host memory: a pinned host tensor is uploaded asynchronously on the
    context's stream (no wait), then stepped and read back into the same pinned tensor; the result
    equals the same step from a device-resident upload, and a pageable upload gives it too."""
    cfg = melt((32, 16, 24), 10, 4, hydro=1, ncg_iters=2, cn_sweeps=4)
    phi, U, dn = random_state(cfg, 95)
    outs = []
    for mode in ("device", "pinned", "pageable"):
        ctx = dscf.Context(cfg, dscf.FP32)
        ctx.set(dscf.U, torch.from_numpy(U).float().cuda())
        ctx.set(dscf.POP, torch.from_numpy(dn).float().cuda())
        host = torch.from_numpy(phi).float()
        if mode == "device":
            ctx.set(dscf.PHI, host.cuda())
        elif mode == "pinned":
            host = host.pin_memory()
            ctx.set(dscf.PHI, host)
        else:
            ctx.set(dscf.PHI, host)
        ctx.step(2)
        out = torch.empty(host.shape, dtype=torch.float32).pin_memory()
        ctx.get_host(dscf.PHI, out)
        ctx.status()
        outs.append(out.numpy().copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
