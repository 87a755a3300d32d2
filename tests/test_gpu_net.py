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
