"""Seeded synthetic inputs and named workloads.

This module holds no arithmetic of the method: it only draws seeded random numbers and
assembles plain parameter dictionaries.  Both the CUDA path (through the binding) and the
FP64 oracle (in the tests) receive exactly the arrays produced here.

Random numbers: a counter-based SplitMix64 stream (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) turned into normal deviates by the
Box-Muller transform, so the same (seed, index) gives the same number on any machine.

Workloads (synthetic stand-ins for the paper's quenched melts and solutions, Sec. 3), all at
dt = 0.1 tau:
  melt32      AB melt f=0.5, chi N=20, 32^3, N=32, tau_s=tau_b=1, noise 0.01, 200 steps
  melt128     AB melt f=0.3, chi N=25, 128^3, N=64, noise 0.01 (tau_s, tau_b chosen from
              {0.6,1,2} x {0.8,1.5})
  batch48     48 melts: 24 at 48^3, 16 at 64^3, 8 at 96^3 with f, chi N, N, seeds and
              viscosities cycled
  solution128 A-B diblock in solvent: phi_p=0.12, f=0.3, chi_AB N=30, chi_BS N=35,
              chi_AS=0, 128^3, N=48, tau_s=0.8, tau_b=1.2, noise 0.005
  melt256     AB melt f=0.5, chi N=20, 256^3, N=64 (learned-predictor workload)
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64: element k is mix(seed + (offset + k + 1) * golden)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the SplitMix64 stream."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller, one per pair of uniforms."""
    u = uniform01(seed, 2 * count)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def n_A(f: float, N: int) -> int:
    """A-block length: f*N rounded to nearest, ties up."""
    return int(np.floor(f * N + 0.5))


def melt(grid, N, f, chiN, tau_s=1.0, tau_b=1.0, noise=0.01, seed=1, dt=0.2, hydro=1,
         ncg_iters=4, cn_sweeps=8, name="melt"):
    nA = n_A(f, N)
    return {
        "name": name, "grid": tuple(int(g) for g in grid), "ns": 2, "N": int(N), "nA": nA,
        "phi_p": 1.0, "chi": {(0, 1): chiN / N}, "kappa": 10.0, "a": 1.1543,
        "dt": dt, "M": 1.0, "tau_s": tau_s, "tau_b": tau_b, "rho0": 1.0, "hydro": hydro,
        "ncg_iters": ncg_iters, "cn_sweeps": cn_sweeps, "phi_floor": 1e-6,
        "noise": noise, "seed": seed,
    }


def solution(grid, N, f, phi_p, chiN_AB, chiN_BS, chiN_AS=0.0, tau_s=0.8, tau_b=1.2,
             noise=0.005, seed=4, dt=0.2, hydro=1, ncg_iters=4, cn_sweeps=8, name="solution"):
    nA = n_A(f, N)
    return {
        "name": name, "grid": tuple(int(g) for g in grid), "ns": 3, "N": int(N), "nA": nA,
        "phi_p": phi_p, "chi": {(0, 1): chiN_AB / N, (1, 2): chiN_BS / N, (0, 2): chiN_AS / N},
        "kappa": 10.0, "a": 1.1543, "dt": dt, "M": 1.0, "tau_s": tau_s, "tau_b": tau_b,
        "rho0": 1.0, "hydro": hydro, "ncg_iters": ncg_iters, "cn_sweeps": cn_sweeps,
        "phi_floor": 1e-6, "noise": noise, "seed": seed,
    }


WORKLOAD_DT = 0.1   # tau: the coupled explicit scheme's velocity stays bounded over long runs


def workload(name: str, **over):
    dt = WORKLOAD_DT
    if name == "melt32":
        cfg = melt((32, 32, 32), 32, 0.5, 20.0, 1.0, 1.0, 0.01, 1, dt=dt, name=name)
    elif name == "melt128":
        cfg = melt((128, 128, 128), 64, 0.3, 25.0, 1.0, 0.8, 0.01, 11, dt=dt, name=name)
    elif name == "solution128":
        cfg = solution((128, 128, 128), 48, 0.3, 0.12, 30.0, 35.0, 0.0, dt=dt, name=name)
    elif name == "melt256":
        cfg = melt((256, 256, 256), 64, 0.5, 20.0, 1.0, 1.0, 0.01, 5, dt=dt, name=name)
    else:
        raise KeyError(name)
    cfg.update(over)
    return cfg


def batch48(**over):
    """The 48 mixed-size replicas: sizes 24 x 48^3, 16 x 64^3, 8 x 96^3; f, chi N and N cycle
    through {0.3, 0.4, 0.5}, {15, 20, 30}, {32, 48, 64}; tau_s through {0.6, 1, 2}, tau_b through
    {0.8, 1.5}; seed 100 + r."""
    sizes = [48] * 24 + [64] * 16 + [96] * 8
    fs, chis, Ns = [0.3, 0.4, 0.5], [15.0, 20.0, 30.0], [32, 48, 64]
    tss, tbs = [0.6, 1.0, 2.0], [0.8, 1.5]
    reps = []
    for r, L in enumerate(sizes):
        cfg = melt((L, L, L), Ns[r % 3], fs[r % 3], chis[(r // 3) % 3], tss[r % 3], tbs[r % 2],
                   0.01, 100 + r, dt=WORKLOAD_DT, name=f"batch48[{r}]")
        cfg.update(over)
        reps.append(cfg)
    return reps


def initial_fields(cfg) -> np.ndarray:
    """Initial compositions [ns, nz, ny, nx] (FP64): homogeneous state plus seeded Gaussian
    noise of standard deviation cfg['noise'] with its mean removed.
    Melt: phi_A = f phi_p + xi, phi_B = (1-f) phi_p - xi.
    Solution: the copolymer fraction phi_p + xi is split f : (1-f) into A and B, and the
    solvent takes the rest."""
    nx, ny, nz = cfg["grid"]
    V = nx * ny * nz
    xi = cfg.get("noise", 0.0) * normal(cfg.get("seed", 1), V)
    xi = xi - xi.mean()
    xi = xi.reshape(nz, ny, nx)
    f = cfg["nA"] / cfg["N"]
    if cfg.get("ns", 2) == 2:
        pp = cfg.get("phi_p", 1.0)
        return np.stack([f * pp + xi, (1.0 - f) * pp - xi])
    pp = cfg["phi_p"] + xi
    return np.stack([f * pp, (1.0 - f) * pp, 1.0 - pp])


def random_field(shape, seed: int, scale: float = 1.0, offset: int = 0) -> np.ndarray:
    """Uniform deviates in [-scale, scale) with the given shape (for potentials in tests)."""
    n = int(np.prod(shape))
    return (2.0 * uniform01(seed, n, offset) - 1.0).reshape(shape) * scale
