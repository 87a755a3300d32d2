"""Element-wise parity of the predictor network's tensor-core kernels with the FP64 oracle
convolutions, on inputs for which every rounding the kernels do is exact or reproducible.

The network computes with BF16 operands and FP32 accumulation, so on general data only norms can
be compared.  Here the data are chosen so that the kernels' arithmetic is exact:
  - potentials are small integers with zero mean per sample and species (the network input
    U - <U> is then exact in BF16);
  - the weights of the two hidden layers are 0 or +-16 (sparse), so every pre-activation is a
    multiple of 16 and tanh gives exactly 0 or +-1 after the rounding to BF16 (tanh(16) is within
    1e-13 of 1), and the output weights are 0 or +-k/8 (sparse);
  - every sum the kernels form is then a sum of multiples of a common power of two whose total
    needs fewer than 24 bits, which FP32 accumulates exactly in any order.
The forward output must therefore equal the FP64 oracle's value bit for bit, on the tcgen05 path
and on the mma.sync path: a wrong row, kernel offset or channel anywhere changes some output by a
multiple of 1/8.  For the parameter gradients the loss targets are the forward output minus
+-k/16 (zero sum per sample and species), so the loss gradient is exact in BF16; the output
layer's weight gradient and the hidden layers' bias gradients are exact, and the hidden layers'
weight gradients (BF16 back-propagated signals, reproduced here with the same round-to-nearest-
even) agree within the FP32 accumulation bound K 2^-22 sum|terms| of their K-term sums.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1204_2088_gb300 import build, dscf, inputs

pytestmark = pytest.mark.gpu

GRID = (128, 8, 4)          # nx a multiple of 128 and ny of 8: the tcgen05 forward applies
B = 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dscf.load()


def bf16(a):
    """Round to FP32, then to BF16 (round to nearest, ties to even), as the kernels store."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def sparse(shape, nnz_per_row, values, seed):
    """Weights [cout][cin][125] with nnz_per_row non-zeros per output channel."""
    cout, cin, K = shape
    W = np.zeros(shape)
    pick = inputs.uniform01(seed, cout * nnz_per_row * 2).reshape(cout, nnz_per_row, 2)
    for co in range(cout):
        for j in range(nnz_per_row):
            idx = int(pick[co, j, 0] * cin * K)
            W[co, idx // K, idx % K] = values[int(pick[co, j, 1] * len(values))]
    return W


def paired_integers(n, lo, hi, seed):
    """n values in [lo, hi] with exactly zero sum: half drawn, the other half their negatives,
    in a seeded order."""
    half = (lo + (inputs.uniform01(seed, n // 2) * (hi - lo + 1)).astype(int)).astype(np.float64)
    v = np.concatenate([half, -half])
    return v[np.argsort(inputs.uniform01(seed + 1, n))]


def exact_problem(grid=GRID):
    nx, ny, nz = grid
    V = nx * ny * nz
    U = np.stack([np.stack([paired_integers(V, -3, 3, 500 + 10 * b + c).reshape(nz, ny, nx) for c in range(2)])
                  for b in range(B)])
    W1 = sparse((32, 2, 125), 3, [16.0, -16.0], 601)
    W2 = sparse((32, 32, 125), 12, [16.0, -16.0], 602)
    W3 = sparse((2, 32, 125), 40, [k / 8 for k in (-3, -2, -1, 1, 2, 3)], 603)
    b1, b2, b3 = np.zeros(32), np.zeros(32), np.array([0.25, -0.5])
    return U, [(W1, b1), (W2, b2), (W3, b3)]


def flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def emulate_forward(params, U, phibar, grid=GRID):
    (W1, b1), (W2, b2), (W3, b3) = params
    x = oracle.net_input(U)
    h1 = bf16(np.tanh(oracle.conv3d(grid, B, W1, b1, x)))
    h2 = bf16(np.tanh(oracle.conv3d(grid, B, W2, b2, h1)))
    y = oracle.conv3d(grid, B, W3, b3, h2)
    phi = y - y.mean(axis=(2, 3, 4), keepdims=True) + np.asarray(phibar)[None, :, None, None, None]
    return phi, (x, h1, h2, y)


@pytest.mark.parametrize("grid", [GRID, (256, 8, 4)], ids=["128x8x4", "256x8x4"])
@pytest.mark.parametrize("path", [0, 1], ids=["tcgen05", "mma.sync"])
def test_forward_is_exact(path, grid):
    """Also at two 128-site x tiles per row (the first layer's periodic x neighbours come from the
    other tile)."""
    U, params = exact_problem(grid)
    phibar = [0.5, 0.5]
    ref, (x, h1, h2, y) = emulate_forward(params, U, phibar, grid)
    # the design: pre-activations are multiples of 16, activations exactly 0 or +-1
    assert set(np.unique(h1)) <= {-1.0, 0.0, 1.0} and set(np.unique(h2)) <= {-1.0, 0.0, 1.0}
    assert 0.05 < (h1 == 0).mean() < 0.95 and 0.05 < (h2 == 0).mean() < 0.95
    net = dscf.Net(grid, B, seed=1)
    net.set_params(torch.from_numpy(flat(params)).float())
    net.set_tensor_path(path)
    got = net.forward(torch.from_numpy(U).float(), phibar).cpu().numpy().astype(np.float64)
    net.status()
    assert net.tensor_path() == (2 if path == 0 else 1)
    assert np.array_equal(got, ref), np.abs(got - ref).max()


def test_forward_is_exact_when_ctas_take_several_tiles():
    """At (128, 64, 48) x 2 samples (1536 tiles of 4 rows) the persistent first layer's CTAs take
    several tiles each, alternating staging buffers and accumulator sets: on the exact problem
    the tcgen05 forward equals the mma.sync forward (which the small grids pin to the oracle) bit
    for bit."""
    grid = (128, 64, 48)
    U, params = exact_problem(grid)
    phibar = [0.5, 0.5]
    net = dscf.Net(grid, B, seed=1)
    net.set_params(torch.from_numpy(flat(params)).float())
    got = []
    for path in (0, 1):
        net.set_tensor_path(path)
        got.append(net.forward(torch.from_numpy(U).float(), phibar).cpu().numpy().astype(np.float64))
        net.status()
    assert np.array_equal(got[0], got[1]), np.abs(got[0] - got[1]).max()
    assert np.abs(got[0]).max() > 0.1


@pytest.mark.parametrize("path", [0, 1], ids=["tcgen05", "mma.sync"])
def test_parameter_gradients_elementwise(path):
    U, params = exact_problem()
    (W1, b1), (W2, b2), (W3, b3) = params
    phibar = [0.5, 0.5]
    phi, (x, h1, h2, y) = emulate_forward(params, U, phibar)
    nx, ny, nz = GRID
    V = nx * ny * nz
    t = np.stack([np.stack([paired_integers(V, 1, 7, 700 + 10 * b + c).reshape(nz, ny, nx) for c in range(2)])
                  for b in range(B)])
    t = (2 * t - np.sign(t)) / 16.0          # odd multiples of 1/16, never zero, zero sum
    tgt = phi - t
    n = phi.size
    # back-propagation with the kernels' BF16 rounding points
    dy = bf16(t / n - (t / n).mean(axis=(2, 3, 4), keepdims=True))
    dW3, _, dh2 = oracle.conv3d_bwd(GRID, B, W3, h2, dy)
    dz2f = dh2 * (1.0 - h2 * h2)
    assert np.array_equal(dz2f.astype(np.float32).astype(np.float64), dz2f)   # exact in FP32
    dz2 = bf16(dz2f)
    db2 = dz2f.sum(axis=(0, 2, 3, 4))
    dW2, _, dh1 = oracle.conv3d_bwd(GRID, B, W2, h1, dz2)
    dz1f = dh1 * (1.0 - h1 * h1)
    assert np.array_equal(dz1f.astype(np.float32).astype(np.float64), dz1f)
    dz1 = bf16(dz1f)
    db1 = dz1f.sum(axis=(0, 2, 3, 4))
    dW1, _, _ = oracle.conv3d_bwd(GRID, B, W1, x, dz1, want_din=False)
    # sum |terms| of each weight-gradient sum, for the accumulation bound
    aW2 = oracle.conv3d_bwd(GRID, B, np.abs(W2), np.abs(h1), np.abs(dz2), want_din=False)[0]
    aW1 = oracle.conv3d_bwd(GRID, B, np.abs(W1), np.abs(x), np.abs(dz1), want_din=False)[0]
    K = B * V

    net = dscf.Net(GRID, B, seed=1)
    net.set_params(torch.from_numpy(flat(params)).float())
    net.set_tensor_path(path)
    loss, g = net.gradient(torch.from_numpy(U).float(), torch.from_numpy(tgt).float(), phibar)
    net.status()
    assert loss == 0.5 * float((t * t).sum()) / n
    (gW1, gb1), (gW2, gb2), (gW3, gb3) = dscf.net_params_split(g.cpu().numpy())
    assert np.array_equal(gW3, dW3)
    assert np.abs(dW3).max() > 0
    assert np.all(gb3 == 0.0)
    assert np.array_equal(gb2, db2) and np.array_equal(gb1, db1)
    for got, ref, a in ((gW2, dW2, aW2), (gW1, dW1, aW1)):
        bound = K * 2.0 ** -22 * a
        assert np.all(np.abs(got - ref) <= bound), np.abs(got - ref).max()
        assert np.abs(ref).max() > 0
