"""Learned density-map predictor on BF16 tensor cores against the FP64 oracle network.

Forward pass and parameter gradients agree with the FP64 reference within the BF16 bound
(activations and weights rounded to 8 mantissa bits, FP32 accumulation); GPU training on pairs
(U, phi[U]) produced by the library's own density map lowers the loss.
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


def rel_l2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def test_forward_matches_fp64_network():
    grid, B = (16, 8, 6), 2
    net = dscf.Net(grid, B, seed=3)
    params = dscf.net_params_split(net.get_params().cpu().numpy())
    nx, ny, nz = grid
    U = inputs.random_field((B, 2, nz, ny, nx), seed=201, scale=0.6)
    phibar = [0.3, 0.7]
    got = net.forward(torch.from_numpy(U).float(), phibar).cpu().numpy()
    ref, _ = oracle.net_forward(grid, params, U.astype(np.float32).astype(np.float64), phibar)
    dev = ref - np.array(phibar)[None, :, None, None, None]
    assert np.abs(got.reshape(B, 2, -1).mean(2) - np.array(phibar)[None]).max() < 1e-6   # exact block masses
    assert rel_l2(got - np.array(phibar)[None, :, None, None, None], dev) < 3e-2


def test_gradient_matches_fp64_network():
    grid, B = (16, 6, 5), 2
    net = dscf.Net(grid, B, seed=4)
    params = dscf.net_params_split(net.get_params().cpu().numpy())
    nx, ny, nz = grid
    U = inputs.random_field((B, 2, nz, ny, nx), seed=211, scale=0.6)
    tgt = np.array([0.3, 0.7])[None, :, None, None, None] + 0.05 * inputs.random_field((B, 2, nz, ny, nx), seed=212)
    phibar = [0.3, 0.7]
    loss, g = net.gradient(torch.from_numpy(U).float(), torch.from_numpy(tgt).float(), phibar)
    rloss, rgrads = oracle.net_loss_grad(grid, params, U.astype(np.float32).astype(np.float64), tgt, phibar)
    assert abs(loss - rloss) < 2e-2 * rloss
    gs = dscf.net_params_split(g.cpu().numpy())
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(gs, rgrads)):
        assert rel_l2(gW, rW) < 6e-2
        if l < 2:
            # a bias gradient is a sum over all sites with strong cancellation (terms ~10x the
            # sum), so the BF16 rounding of the backpropagated signal shows up ~10x amplified
            assert rel_l2(gb, rb) < 1.5e-1
        else:   # the output bias cannot change phi_hat (mean removal): its gradient is zero
            assert np.abs(gb).max() < 1e-3 * np.abs(rW).max() and np.abs(rb).max() < 1e-12


def test_training_on_method_generated_pairs_lowers_the_loss():
    """Pairs (U, phi[U]) from the library's exact density map on a small melt; Adam on GPU."""
    cfg = inputs.melt((16, 16, 16), 8, 0.5, 10.0)
    cfg["nA"] = 4
    ctx = dscf.Context(cfg, dscf.FP32)
    B = 4
    net = dscf.Net(cfg["grid"], B, seed=5)
    phibar = [0.5, 0.5]
    Us, Ps = [], []
    for k in range(B):
        # smooth random potentials: a few low Fourier modes
        z, y, x = np.meshgrid(*(np.arange(16),) * 3, indexing="ij")
        U = np.zeros((2, 16, 16, 16))
        for m in range(4):
            kv = 2 * np.pi * inputs.uniform01(300 + 10 * k + m, 3) * 2 / 16
            ph = inputs.uniform01(400 + 10 * k + m, 2)
            U[0] += 0.4 * np.cos(kv[0] * x + kv[1] * y + kv[2] * z + 6.28 * ph[0])
            U[1] -= 0.4 * np.cos(kv[0] * x + kv[1] * y + kv[2] * z + 6.28 * ph[1])
        Ut = torch.from_numpy(U).float().cuda()
        Us.append(Ut)
        Ps.append(ctx.densities(Ut))
    U = torch.stack(Us)
    P = torch.stack(Ps)
    first = net.train_step(U, P, phibar, lr=2e-3, want_loss=True)
    for _ in range(150):
        net.train_step(U, P, phibar, lr=2e-3)
    last = net.train_step(U, P, phibar, lr=2e-3, want_loss=True)
    assert last < 0.2 * first


def _melt32(N=16, seed=31):
    cfg = inputs.melt((32, 16, 12), N, 0.5, 15.0, seed=seed, noise=0.03)
    return cfg


def _ctx_from(cfg, phi0):
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set(dscf.PHI, torch.from_numpy(phi0).float().cuda())
    return ctx


def test_predictor_that_never_passes_falls_back_to_the_exact_path_bitwise():
    cfg = _melt32()
    phi0 = inputs.initial_fields(cfg)
    ref = _ctx_from(cfg, phi0)
    ctx = _ctx_from(cfg, phi0)
    net = dscf.Net(cfg["grid"], 1, seed=7)           # untrained: far outside any tolerance
    ctx.set_predictor(net, corrector_every=2, tol=1e-9)
    ref.step(5)
    ctx.step(5)
    for f in (dscf.PHI, dscf.U, dscf.POP, dscf.PHIM):
        assert torch.equal(ctx.get(f), ref.get(f)), f
    d = ctx.diagnostics()
    assert d["pred_steps"] == 0 and d["exact_steps"] == 5 and d["pred_err"] > 1e-9


def test_predictor_steps_use_the_network_and_the_corrector_judges_it():
    cfg = _melt32()
    phi0 = inputs.initial_fields(cfg)
    phibar = [cfg["nA"] / cfg["N"], 1 - cfg["nA"] / cfg["N"]]
    ctx = _ctx_from(cfg, phi0)
    net = dscf.Net(cfg["grid"], 1, seed=8)
    ctx.set_predictor(net, corrector_every=2, tol=1e3, ncg_iters=2)   # always accepted
    ctx.step(1)                      # exact step; first judgement: the network's own error
    d = ctx.diagnostics()
    assert d["exact_steps"] == 1 and d["pred_steps"] == 0
    U = ctx.get(dscf.U)
    exact = ctx.densities(U)
    pred = net.forward(U[None], phibar)[0]
    torch.cuda.synchronize()
    assert abs(d["pred_err"] - (pred - exact).abs().max().item()) < 1e-6
    ctx.step(1)                      # predictor step
    d = ctx.diagnostics()
    assert d["exact_steps"] == 1 and d["pred_steps"] == 1 and d["ncg_iters"] == 2
    # after a predictor step the inversion's density is the network at the committed potential
    U = ctx.get(dscf.U)
    pred = net.forward(U[None], phibar)[0]
    torch.cuda.synchronize()
    assert (ctx.get(dscf.PHIM) - pred).abs().max().item() < 1e-5
    # masses stay exact through the convection-diffusion update
    m0 = phi0.astype(np.float32).astype(np.float64).reshape(2, -1).sum(1)
    phi = ctx.get(dscf.PHI)
    assert np.abs(phi.double().cpu().numpy().reshape(2, -1).sum(1) - m0).max() < 1e-6 * m0.max()
    # the corrector after a predictor step judges it by ||phi[U] - phi*||_inf at its potential
    want = (phi - ctx.densities(U)).abs().max().item()
    ctx.step(1)
    d = ctx.diagnostics()
    assert d["exact_steps"] == 2 and d["pred_steps"] == 1 and d["ncg_iters"] == cfg["ncg_iters"]
    assert abs(d["pred_err"] - want) < 1e-6 * max(1.0, want)
    ctx.step(1)                      # predictor step again
    # detaching returns to the exact path, starting from the exact density of the current state:
    # the next step agrees with that of a fresh context given the same fields (which differs only
    # in its reference masses, taken from the fields it was given, and its stored velocity)
    ctx.set_predictor(None)
    fresh = dscf.Context(cfg, dscf.FP32)
    for f in (dscf.PHI, dscf.U, dscf.POP):
        fresh.set(f, ctx.get(f))
    ctx.step(1)
    fresh.step(1)
    for f in (dscf.PHI, dscf.U):
        a, b = ctx.get(f), fresh.get(f)
        r = ((a - b).abs().max() / b.abs().max()).item()
        assert r < 1e-4, (f, r)


def test_corrector_schedule():
    """Exact steps at counters 0, k, 2k, ...; between them the predictor runs exactly when the
    last judgement passed (an untrained network can fail it: its steps may even go non-finite)."""
    cfg = _melt32()
    ctx = _ctx_from(cfg, inputs.initial_fields(cfg))
    tol = 1e3
    ctx.set_predictor(dscf.Net(cfg["grid"], 1, seed=8), corrector_every=3, tol=tol)
    ok = None
    d = ctx.diagnostics()
    for i in range(7):
        ctx.step(1)
        e = ctx.diagnostics()
        took_pred = e["pred_steps"] > d["pred_steps"]
        assert e["pred_steps"] + e["exact_steps"] == i + 1
        if i % 3 == 0:
            assert not took_pred
            ok = bool(np.isfinite(e["pred_err"]) and e["pred_err"] <= tol)
        else:
            assert took_pred == ok, (i, e)
        d = e
    assert d["steps"] == 7


def test_predictor_rejects_unsupported_contexts():
    cfg = _melt32()
    net = dscf.Net(cfg["grid"], 1, seed=9)
    with pytest.raises(dscf.DSCFError):
        dscf.Context(cfg, dscf.FP64).set_predictor(net)
    with pytest.raises(dscf.DSCFError):
        dscf.Context(cfg, dscf.FP32).set_predictor(dscf.Net((16, 16, 12), 1))
    with pytest.raises(dscf.DSCFError):
        dscf.Context(cfg, dscf.FP32).set_predictor(dscf.Net(cfg["grid"], 2))
    with pytest.raises(dscf.DSCFError):
        dscf.Context(cfg, dscf.FP32).set_predictor(net, corrector_every=0)
    with pytest.raises(dscf.DSCFError):
        dscf.Context(cfg, dscf.FP32).set_predictor(net, ncg_iters=33)


def _events_ms(fn, reps):
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def test_trained_predictor_gain_over_the_exact_method():
    """What a network trained on the method's own (U, phi[U]) pairs gains, measured honestly.

    Symmetric melt f = 0.5, chi N = 20, N = 32 on 32^3 (FP32).  The exact run supplies the
    pairs of its first 120 steps; the network (BF16 kernels, Adam on the GPU) is judged on the
    later 40.  Then, from the exact state at step 120, 40 steps with the predictor attached
    (exact corrector every 10 steps, fallback above tol) against 40 exact steps: the run must
    take predictor steps, stay finite and close to the exact trajectory, and be faster."""
    cfg = inputs.melt((32, 32, 32), 32, 0.5, 20.0, seed=1)
    phibar = [cfg["nA"] / cfg["N"], 1 - cfg["nA"] / cfg["N"]]
    ctx = dscf.Context(cfg, dscf.FP32)
    ctx.set(dscf.PHI, torch.from_numpy(inputs.initial_fields(cfg)).float().cuda())
    T0, T = 120, 160
    Us, Ps = [], []
    for t in range(1, T + 1):
        ctx.step(1)
        Us.append(ctx.get(dscf.U).clone())
        Ps.append(ctx.get(dscf.PHIM).clone())     # phi[U] of the step's inverted potential
        if t == T0:
            state = {f: ctx.get(f).clone() for f in (dscf.PHI, dscf.U, dscf.POP)}
    phi_exact = ctx.get(dscf.PHI)
    U, P = torch.stack(Us), torch.stack(Ps)

    B, iters = 8, 2000
    net = dscf.Net(cfg["grid"], B, seed=3)
    one = dscf.Net(cfg["grid"], 1, seed=3)

    def held_out_err():
        return max((one.forward(U[t:t + 1], phibar)[0] - P[t]).abs().max().item() for t in range(T0, T, 5))

    e0 = held_out_err()
    g = torch.Generator().manual_seed(0)
    for it in range(iters):
        idx = torch.randint(0, T0, (B,), generator=g)
        net.train_step(U[idx], P[idx], phibar, lr=3e-4 * 0.5 * (1 + np.cos(np.pi * it / iters)) + 1e-6)
    one.set_params(net.get_params())
    e1 = held_out_err()
    assert e1 < 0.1 * e0 and e1 < 3e-3, (e0, e1)

    tol = 3e-3
    pred = dscf.Context(cfg, dscf.FP32)
    ref = dscf.Context(cfg, dscf.FP32)
    for c in (pred, ref):
        for f, v in state.items():
            c.set(f, v)
    pred.set_predictor(one, corrector_every=10, tol=tol, ncg_iters=1)
    t_pred = _events_ms(lambda: pred.step(T - T0), 1)
    t_ref = _events_ms(lambda: ref.step(T - T0), 1)
    d = pred.diagnostics()
    phi = pred.get(dscf.PHI)
    dev = (phi - ref.get(dscf.PHI)).abs().max().item()
    # a context restarted from the fields reproduces the continued run up to FP32 rounding
    assert (ref.get(dscf.PHI) - phi_exact).abs().max().item() < 1e-4
    assert d["pred_steps"] > 0 and d["pred_steps"] + d["exact_steps"] == T - T0
    assert torch.isfinite(phi).all()
    assert dev < 2 * tol, dev
    assert t_ref / t_pred > 1.1, (t_ref, t_pred, d)


def test_tcgen05_forward_matches_mma_sync_and_fp64_network():
    """Forward convolutions on tcgen05 (operands in shared memory, accumulators in tensor memory)
    on a 128-wide grid: the same network on the warp-level mma.sync path agrees up to FP32
    summation order and the BF16 rounding it can flip, and both match the FP64 CPU network within
    the BF16 bound."""
    grid, B = (128, 8, 6), 2
    net = dscf.Net(grid, B, seed=13)
    assert net.tensor_path() == 2
    params = dscf.net_params_split(net.get_params().cpu().numpy())
    nx, ny, nz = grid
    U = inputs.random_field((B, 2, nz, ny, nx), seed=301, scale=0.6)
    phibar = [0.3, 0.7]
    Ut = torch.from_numpy(U).float()
    tc = net.forward(Ut, phibar).cpu().numpy()
    net.status()
    net.set_tensor_path(1)
    assert net.tensor_path() == 1
    ms = net.forward(Ut, phibar).cpu().numpy()
    net.set_tensor_path(0)
    pb = np.array(phibar)[None, :, None, None, None]
    dev = ms - pb
    assert np.abs(tc - ms).max() < 2e-2 * np.abs(dev).max(), np.abs(tc - ms).max()
    assert rel_l2(tc - pb, dev) < 2e-3
    ref, _ = oracle.net_forward(grid, params, U.astype(np.float32).astype(np.float64), phibar)
    assert rel_l2(tc - pb, ref - pb) < 3e-2
    assert np.abs(tc.reshape(B, 2, -1).mean(2) - np.array(phibar)[None]).max() < 1e-6


def test_tcgen05_training_forward_gives_the_same_gradient():
    """Training at a 128-wide grid runs its forward pass on tcgen05; the gradient agrees with the
    one taken with the mma.sync forward."""
    grid, B = (128, 8, 4), 1
    net = dscf.Net(grid, B, seed=14)
    assert net.tensor_path() == 2
    nx, ny, nz = grid
    U = torch.from_numpy(inputs.random_field((B, 2, nz, ny, nx), seed=311, scale=0.6)).float()
    tgt = torch.from_numpy(np.array([0.4, 0.6])[None, :, None, None, None]
                           + 0.05 * inputs.random_field((B, 2, nz, ny, nx), seed=312)).float()
    l0, g0 = net.gradient(U, tgt, [0.4, 0.6])
    net.status()
    net.set_tensor_path(1)
    l1, g1 = net.gradient(U, tgt, [0.4, 0.6])
    assert abs(l0 - l1) < 1e-3 * l1
    assert rel_l2(g0.cpu().numpy(), g1.cpu().numpy()) < 2e-2
