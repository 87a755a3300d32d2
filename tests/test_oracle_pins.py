"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: a closed form, a
library routine used as an independent route (FFT convolution), brute-force enumeration of
chain conformations (Eq. 2 taken literally), a finite-difference derivative, a conservation
law, or a value the paper prints.  A plausible slip in the oracle (a dropped term, a wrong
index or sign, a transposed operand) fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1204_2088_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cfg_small(grid=(5, 6, 7), N=6, nA=2, chi=0.4, ns=2, phi_p=1.0, **kw):
    c = inputs.melt(grid, N, 0.5, chi * N, **kw)
    c["nA"] = nA
    if ns == 3:
        c["ns"] = 3
        c["phi_p"] = phi_p
        c["chi"] = {(0, 1): chi, (1, 2): 1.3 * chi, (0, 2): 0.2 * chi}
    return c


def symbol(a, kvec):
    """Fourier symbol of the separable moment-matched 27-point stencil."""
    al = a * a / 6.0
    return np.prod([1.0 - 2.0 * al + 2.0 * al * np.cos(k) for k in kvec])


def kgrid(grid):
    nx, ny, nz = grid
    kz, ky, kx = np.meshgrid(2 * np.pi * np.fft.fftfreq(nz), 2 * np.pi * np.fft.fftfreq(ny),
                             2 * np.pi * np.fft.fftfreq(nx), indexing="ij")
    return kx, ky, kz


# ---------------------------------------------------------------------------------------------
# Linkage operator (Eq. 17 and the Gaussian kernel after it)
# ---------------------------------------------------------------------------------------------
def test_stencil_normalised_and_moment_matched():
    a = 1.1543
    w = oracle.stencil_weights(a)
    counts = np.array([1, 6, 12, 8])
    assert abs((counts * w).sum() - 1.0) < 1e-15            # sigma[1] = 1
    # second moment along x: faces +-x (2), edges with x (8), corners (8)
    m2 = 2 * w[1] + 8 * w[2] + 8 * w[3]
    assert abs(m2 - a * a / 3.0) < 1e-15                     # per-axis variance of a Gaussian bond


def test_sigma_plane_wave_closed_form():
    cfg = cfg_small(grid=(5, 6, 7))
    nx, ny, nz = cfg["grid"]
    k = (2 * np.pi * 1 / nx, 2 * np.pi * 2 / ny, 2 * np.pi * 3 / nz)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.cos(k[0] * x + k[1] * y + k[2] * z + 0.3)
    out = oracle.sigma(cfg, f)
    assert np.abs(out - symbol(cfg["a"], k) * f).max() < 1e-14


def test_sigma_equals_fft_convolution():
    cfg = cfg_small(grid=(4, 7, 3))   # nx=4, tiny nz=3: periodic wrap on both sides
    f = inputs.random_field((3, 7, 4), seed=3)
    kx, ky, kz = kgrid(cfg["grid"])
    al = cfg["a"] ** 2 / 6.0
    sym = (1 - 2 * al + 2 * al * np.cos(kx)) * (1 - 2 * al + 2 * al * np.cos(ky)) * (1 - 2 * al + 2 * al * np.cos(kz))
    ref = np.real(np.fft.ifftn(np.fft.fftn(f) * sym))
    assert np.abs(oracle.sigma(cfg, f) - ref).max() < 1e-14


# ---------------------------------------------------------------------------------------------
# Propagators, densities, Q (Eq. 2, 16, 17)
# ---------------------------------------------------------------------------------------------
def test_homogeneous_field_propagator_is_exponential():
    cfg = cfg_small(grid=(4, 5, 6), N=7, nA=3)
    wA, wB = 0.37, -0.21
    U = np.stack([np.full((6, 5, 4), wA), np.full((6, 5, 4), wB)])
    phi, Q, _, G = oracle.densities(cfg, U, want_stack=True)
    for s in range(cfg["N"] + 1):
        expo = wA * min(s, 3) + wB * max(s - 3, 0)
        assert np.abs(G[s] - np.exp(-expo)).max() < 1e-14 * max(1.0, np.exp(-expo))
    assert abs(Q - np.exp(-(3 * wA + 4 * wB))) < 1e-14
    assert np.abs(phi[0] - 3 / 7).max() < 1e-14 and np.abs(phi[1] - 4 / 7).max() < 1e-14


def brute_force_densities(cfg, U):
    """Eq. 2 taken literally on a tiny lattice: sum over all bead-position paths
    R_1..R_N of prod_s exp(-U_{I_s}(R_s)) prod_bonds T(R_s - R_{s-1}), where T is the
    27-point Gaussian bond weight built here from the stencil offsets."""
    nx, ny, nz = cfg["grid"]
    V = nx * ny * nz
    al = cfg["a"] ** 2 / 6.0
    w1 = {-1: al, 0: 1 - 2 * al, 1: al}
    T = np.zeros((V, V))
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        r = x + nx * (y + ny * z)
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            r2 = (x + dx) % nx + nx * (((y + dy) % ny) + ny * ((z + dz) % nz))
            T[r, r2] += w1[dx] * w1[dy] * w1[dz]
    N, nA = cfg["N"], cfg["nA"]
    B = [np.exp(-U[0].reshape(-1)) if s < nA else np.exp(-U[1].reshape(-1)) for s in range(N)]
    # W[r1,...,rN]
    W = B[0].copy()
    for s in range(1, N):
        W = W[..., None] * T.reshape((1,) * (s - 1) + (V, V)) * B[s].reshape((1,) * s + (V,))
    Phi = W.sum()
    marg = [W.sum(axis=tuple(a for a in range(N) if a != s)) for s in range(N)]
    pref = cfg["phi_p"] * V / (N * Phi)
    phiA = pref * sum(marg[s] for s in range(nA))
    phiB = pref * sum(marg[s] for s in range(nA, N))
    return np.stack([phiA, phiB]).reshape(2, nz, ny, nx), Phi / V


@pytest.mark.parametrize("grid,N,nA", [((2, 3, 2), 4, 2), ((3, 2, 2), 3, 1), ((1, 3, 4), 4, 3)])
def test_densities_brute_force_paths(grid, N, nA):
    cfg = cfg_small(grid=grid, N=N, nA=nA)
    nx, ny, nz = grid
    U = inputs.random_field((2, nz, ny, nx), seed=11 + N, scale=0.7)
    phi, Q, _ = oracle.densities(cfg, U)
    ref, Qref = brute_force_densities(cfg, U)
    assert abs(Q - Qref) < 1e-13 * Qref
    assert np.abs(phi - ref).max() < 1e-13


def test_block_masses_and_solvent():
    cfg = cfg_small(grid=(6, 5, 4), N=9, nA=4, ns=3, phi_p=0.3)
    U = inputs.random_field((3, 4, 5, 6), seed=5, scale=0.8)
    phi, Q, qs = oracle.densities(cfg, U)
    V = 120
    assert abs(phi[0].sum() - V * 0.3 * 4 / 9) < 1e-12
    assert abs(phi[1].sum() - V * 0.3 * 5 / 9) < 1e-12
    es = np.exp(-U[2])
    assert abs(qs - es.mean()) < 1e-14
    assert np.abs(phi[2] - 0.7 * es / es.mean()).max() < 1e-14


# ---------------------------------------------------------------------------------------------
# Self-consistent inversion (Fletcher-Reeves NCG on the Legendre functional)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("ns", [2, 3])
def test_objective_gradient_is_density_deficit(ns):
    cfg = cfg_small(grid=(4, 3, 5), N=5, nA=2, ns=ns, phi_p=0.4)
    shp = (ns, 5, 3, 4)
    U = inputs.random_field(shp, seed=21, scale=0.5)
    target = 0.2 + 0.1 * inputs.uniform01(22, int(np.prod(shp))).reshape(shp)
    phi, _, _ = oracle.densities(cfg, U)
    grad = target - phi
    h = 1e-5
    for (I, z, y, x) in [(0, 0, 0, 0), (1, 4, 2, 3), (ns - 1, 2, 1, 1), (0, 3, 0, 2)]:
        Up = U.copy(); Up[I, z, y, x] += h
        Um = U.copy(); Um[I, z, y, x] -= h
        fd = (oracle.objective(cfg, Up, target) - oracle.objective(cfg, Um, target)) / (2 * h)
        assert abs(fd - grad[I, z, y, x]) < 1e-8


def test_ncg_recovers_potentials_up_to_gauge():
    cfg = cfg_small(grid=(4, 4, 3), N=6, nA=3, ncg_iters=300)
    Utrue = inputs.random_field((2, 3, 4, 4), seed=31, scale=0.5)
    target, _, _ = oracle.densities(cfg, Utrue)
    U, phim, info = oracle.ncg(cfg, target, np.zeros_like(Utrue))
    assert np.abs(phim - target).max() < 1e-10
    # the potential is unique up to one constant per species (uniform U_A, U_B are gauges)
    for I in range(2):
        dev = U[I] - Utrue[I]
        assert np.ptp(dev) < 1e-7
    assert info[-1] < 1e-10


def test_ncg_uniform_target_keeps_zero_potential():
    cfg = cfg_small(grid=(3, 3, 3), N=4, nA=2, ncg_iters=3)
    target = np.stack([np.full((3, 3, 3), 0.5), np.full((3, 3, 3), 0.5)])
    U, phim, _ = oracle.ncg(cfg, target, np.zeros_like(target))
    assert np.abs(U).max() < 1e-13
    assert np.abs(phim - 0.5).max() < 1e-14


def _residual_history(info, K):
    """max|g| at the start of iterations 0..K (info layout of oracle.ncg)."""
    return [info[1]] + [info[2 + 4 * k + 3] for k in range(K)]


def test_ncg_tolerance_stop_is_a_truncated_fixed_count_run():
    cfg = cfg_small(grid=(4, 5, 3), N=6, nA=3, ncg_iters=8)
    Utrue = inputs.random_field((2, 3, 5, 4), seed=33, scale=0.4)
    target, _, _ = oracle.densities(cfg, Utrue)
    U0 = np.zeros_like(Utrue)
    _, _, info_full = oracle.ncg(cfg, target, U0)
    r = _residual_history(info_full, 8)
    j = 3
    assert min(r[:j]) > 1.01 * r[j]
    tol = 1.005 * r[j]
    Ut, pt, info_t, k = oracle.ncg_run(dict(cfg, ncg_tol=tol), target, U0)
    Uf, pf, info_f, kf = oracle.ncg_run(dict(cfg, ncg_iters=j), target, U0)
    assert k == j and kf == j
    assert np.array_equal(Ut, Uf) and np.array_equal(pt, pf)
    assert np.array_equal(info_t[:2 + 4 * j], info_f)
    assert np.all(info_t[2 + 4 * j:] == 0.0)   # iterations not run leave their entries untouched


def test_ncg_tolerance_above_the_start_residual_runs_no_iteration():
    cfg = cfg_small(grid=(3, 4, 3), N=4, nA=2, ncg_iters=5)
    target = 0.5 + 0.05 * inputs.random_field((2, 3, 4, 3), seed=35, scale=1.0)
    U0 = inputs.random_field((2, 3, 4, 3), seed=36, scale=0.1)
    phi0, _, _ = oracle.densities(cfg, U0)
    gmax0 = np.abs(target - phi0).max()
    U, phim, info, k = oracle.ncg_run(dict(cfg, ncg_tol=1.5 * gmax0), target, U0)
    assert k == 0
    assert np.array_equal(U, U0)
    assert np.abs(phim - phi0).max() < 1e-15
    assert abs(info[1] - gmax0) < 1e-15


def test_ncg_tolerance_stop_meets_the_tolerance():
    cfg = dict(cfg_small(grid=(4, 4, 3), N=6, nA=3, ncg_iters=300), ncg_tol=1e-9)
    Utrue = inputs.random_field((2, 3, 4, 4), seed=31, scale=0.5)
    target, _, _ = oracle.densities(cfg, Utrue)
    U, phim, info, k = oracle.ncg_run(cfg, target, np.zeros_like(Utrue))
    assert 0 < k < 300
    assert np.abs(phim - target).max() < 1e-9              # the exit residual is the true one
    r = _residual_history(info, k)
    assert r[k] < 1e-9 and min(r[:k]) >= 1e-9               # and it stopped at the first crossing


# ---------------------------------------------------------------------------------------------
# Chemical potential (Eq. 4) and force (Eq. 8)
# ---------------------------------------------------------------------------------------------
def test_mu_uniform_closed_form():
    cfg = cfg_small(grid=(3, 4, 5), chi=0.625)
    phA, phB = 0.37, 0.61
    phi = np.stack([np.full((5, 4, 3), phA), np.full((5, 4, 3), phB)])
    mu = oracle.mu(cfg, np.zeros_like(phi), phi)
    kap = 10.0 * (phA + phB - 1.0)
    assert np.abs(mu[0] - (0.625 * phB + kap)).max() < 1e-14
    assert np.abs(mu[1] - (0.625 * phA + kap)).max() < 1e-14
    assert np.abs((mu[0] - mu[1]) - 0.625 * (phB - phA)).max() < 1e-14


def test_mu_general_against_fft():
    cfg = cfg_small(grid=(6, 5, 4), ns=3, phi_p=0.5, chi=0.3)
    shp = (3, 4, 5, 6)
    U = inputs.random_field(shp, seed=41)
    phi = 0.3 + 0.1 * inputs.random_field(shp, seed=42)
    kx, ky, kz = kgrid(cfg["grid"])
    al = cfg["a"] ** 2 / 6.0
    sym = (1 - 2 * al + 2 * al * np.cos(kx)) * (1 - 2 * al + 2 * al * np.cos(ky)) * (1 - 2 * al + 2 * al * np.cos(kz))
    sphi = np.stack([np.real(np.fft.ifftn(np.fft.fftn(phi[J]) * sym)) for J in range(3)])
    chi = np.zeros((3, 3))
    for (i, j), v in cfg["chi"].items():
        chi[i, j] = chi[j, i] = v
    ref = -U + np.einsum("ij,jzyx->izyx", chi, sphi) + 10.0 * (phi.sum(0) - 1.0)[None]
    assert np.abs(oracle.mu(cfg, U, phi) - ref).max() < 1e-13


def test_force_central_difference_closed_form():
    cfg = cfg_small(grid=(8, 6, 5))
    z, y, x = np.meshgrid(np.arange(5), np.arange(6), np.arange(8), indexing="ij")
    k = 2 * np.pi / 8
    mu = np.stack([np.sin(k * x), 2.0 * np.sin(k * x)])
    phi = np.stack([np.full_like(mu[0], 0.3), np.full_like(mu[0], 0.7)])
    f = oracle.force(cfg, phi, mu)
    ref = -(0.3 + 1.4) * np.sin(k) * np.cos(k * x)     # (sin(k(x+1)) - sin(k(x-1)))/2
    assert np.abs(f[0] - ref).max() < 1e-14
    assert np.abs(f[1]).max() == 0.0 and np.abs(f[2]).max() == 0.0


# ---------------------------------------------------------------------------------------------
# Lattice Boltzmann (Eq. 9-15, Table 1)
# ---------------------------------------------------------------------------------------------
def test_table1_basis_orthogonal_with_paper_weights():
    e, w, b, c = oracle.lb_basis()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - np.eye(3) / 3).max() < 1e-15
    G = np.einsum("i,ki,li->kl", w, e, e)
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-15          # mutually orthogonal
    # norms b_k = sum_i w_i e_ki^2 worked out by hand from Table 1
    hand = np.array([1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 9, 4 / 3, 1 / 9, 1 / 9, 1 / 9,
                     2 / 3, 2 / 3, 2 / 3, 2 / 9, 2 / 9, 2 / 9, 2, 4 / 9, 4 / 3])
    assert np.abs(b - hand).max() < 1e-15
    expect = {(0, 0, 0)}
    for a in range(3):
        for sgn in (1, -1):
            v = [0, 0, 0]; v[a] = sgn
            expect.add(tuple(v))
    for a in range(3):
        for b_ in range(a + 1, 3):
            for sa in (1, -1):
                for sb in (1, -1):
                    v = [0, 0, 0]; v[a] = sa; v[b_] = sb
                    expect.add(tuple(v))
    assert set(map(tuple, c.tolist())) == expect and len(expect) == 19


def test_equilibrium_moment_constraints():
    _, w, _, c = oracle.lb_basis()
    rho, u = 1.07, np.array([0.03, -0.05, 0.02])
    neq = oracle.lb_equilibrium(rho, u)
    assert abs(neq.sum() - rho) < 1e-15
    assert np.abs(neq @ c - rho * u).max() < 1e-15
    P = np.einsum("i,ia,ib->ab", neq, c, c)
    assert np.abs(P - (rho * np.outer(u, u) + rho / 3 * np.eye(3))).max() < 1e-15


def lb_cfg(grid, tau_s=1.0, tau_b=1.0):  # noqa: E302
    return cfg_small(grid=grid, tau_s=tau_s, tau_b=tau_b)


def test_lb_equilibrium_fixed_point_and_conservation():
    grid = (5, 4, 6)
    cfg = lb_cfg(grid, 0.7, 1.3)
    _, w, _, _ = oracle.lb_basis()
    u = np.array([0.02, -0.01, 0.015])
    neq = oracle.lb_equilibrium(1.1, u)
    n = np.broadcast_to(neq[:, None, None, None], (19, 6, 4, 5)).copy()
    out, uo = oracle.lb_step(cfg, n)
    assert np.abs(out - n).max() < 1e-15
    assert np.abs(uo - u[:, None, None, None]).max() < 1e-15
    # random state with random force: mass exact, momentum grows by exactly sum f
    n = w[:, None, None, None] * (1.0 + 0.05 * inputs.random_field((19, 6, 4, 5), seed=51))
    f = 1e-3 * inputs.random_field((3, 6, 4, 5), seed=52)
    _, _, _, c = oracle.lb_basis()
    out, _ = oracle.lb_step(cfg, n, f)
    assert abs(out.sum() - n.sum()) < 1e-12
    j0 = np.einsum("izyx,ia->a", n, c)
    j1 = np.einsum("izyx,ia->a", out, c)
    assert np.abs(j1 - j0 - f.reshape(3, -1).sum(1)).max() < 1e-13


@pytest.mark.parametrize("tau", [0.6, 1.0, 2.0])
def test_shear_wave_decay_gives_kinematic_viscosity(tau):
    """u_x = U0 sin(k z) decays as exp(-nu k^2 t) with nu = c_s^2 (tau - 1/2) (Eq. 15 with
    gamma_s = 1 - 1/tau, lattice units)."""
    L = 96
    cfg = lb_cfg((1, 1, L), tau_s=tau, tau_b=1.0)
    k = 2 * np.pi / L
    z = np.arange(L)
    n = np.stack([oracle.lb_equilibrium(1.0, [1e-4 * np.sin(k * zz), 0, 0]) for zz in z], axis=1)
    n = n.reshape(19, L, 1, 1)
    amps = []
    for t in range(400):
        n, u = oracle.lb_step(cfg, n)
        amps.append(2.0 / L * (u[0, :, 0, 0] * np.sin(k * z)).sum())
    t1, t2 = 100, 399
    rate = -np.log(amps[t2] / amps[t1]) / (t2 - t1)
    nu = (tau - 0.5) / 3.0
    # discrete (lattice) wave number of the second-order scheme: k_hat^2 = 2 - 2 cos k
    assert abs(rate / (nu * (2 - 2 * np.cos(k))) - 1.0) < 2e-3


@pytest.mark.parametrize("tau_b", [0.8, 1.5])
def test_sound_wave_damping_gives_bulk_viscosity(tau_b):
    """A density wave decays with Gamma = k^2 (4 nu/3 + nu_b)/2, nu_b = (2/3) c_s^2 (tau_b - 1/2),
    and oscillates at c_s k."""
    L = 64
    tau_s = 0.9
    cfg = lb_cfg((L, 1, 1), tau_s=tau_s, tau_b=tau_b)
    k = 2 * np.pi / L
    x = np.arange(L)
    n = np.stack([oracle.lb_equilibrium(1.0 + 1e-5 * np.cos(k * xx), [0, 0, 0]) for xx in x], axis=1)
    n = n.reshape(19, 1, 1, L)
    _, _, _, c = oracle.lb_basis()
    T = 600
    rk, jk = [], []
    for t in range(T):
        n, u = oracle.lb_step(cfg, n)
        rho = n.sum(0)[0, 0]
        jx = np.einsum("i,ix->x", c[:, 0].astype(float), n[:, 0, 0, :])
        rk.append(2.0 / L * ((rho - 1.0) * np.cos(k * x)).sum())
        jk.append(2.0 / L * (jx * np.sin(k * x)).sum())
    rk, jk = np.array(rk), np.array(jk)
    E = rk ** 2 / 3.0 + jk ** 2                     # acoustic energy of the mode
    nu, nub = (tau_s - 0.5) / 3.0, 2.0 / 9.0 * (tau_b - 0.5)
    k2 = 2 - 2 * np.cos(k)
    gamma = 0.5 * k2 * (4.0 * nu / 3.0 + nub)
    # average log-energy slope over whole periods
    period = 2 * np.pi / (np.sqrt(k2 / 3.0))
    t1 = int(round(period)); t2 = int(round(5 * period))
    rate = -(np.log(E[t2]) - np.log(E[t1])) / (t2 - t1) / 2.0
    assert abs(rate / gamma - 1.0) < 2e-2
    # frequency: zero crossings of the density amplitude
    s = np.sign(rk)
    crossings = np.nonzero(s[1:] != s[:-1])[0]
    w_meas = np.pi / np.mean(np.diff(crossings))
    assert abs(w_meas / (np.sin(k) / np.sqrt(3.0)) - 1.0) < 3e-2


def test_printed_viscosities_back_solve_to_unit_relaxation():
    """Eq. 15 solved for gamma with the viscosities the paper prints.  With LB mass density 1
    (m0/h^3) the Fig. 2 values (dt = 0.2 tau, eta_s = 0.83, eta_b = 0.56) give gamma_s and
    gamma_b within 0.005 of zero, i.e. relaxation times of one LB step -- the unit convention
    the oracle uses; every printed pair maps to a stable relaxation (|gamma| < 1)."""
    with open(os.path.join(GOLDEN, "viscosity_pins.json")) as fh:
        pins = json.load(fh)["pins"]
    for p in pins:
        dt, rho = p["dt"], 1.0
        cs2 = 1.0 / (3.0 * dt * dt)            # (h/dt)^2 / 3 in h^2/tau^2
        xs = p["eta_s"] / (dt * rho * cs2 / 2.0)
        xb = p["eta_b"] / (dt * rho * cs2 / 3.0)
        gs = (xs - 1.0) / (xs + 1.0)
        gb = (xb - 1.0) / (xb + 1.0)
        assert -1.0 < gs < 1.0 and -1.0 < gb < 1.0
        if p["figure"] == "Fig. 2":
            assert abs(gs) < 5e-3 and abs(gb) < 5e-3
        # the LB relaxation times that reproduce the printed values, tau = 1/(1 - gamma)
        tau_s = 1.0 / (1.0 - gs)
        assert abs(p["eta_s"] - rho * (tau_s - 0.5) / (3.0 * dt)) < 1e-12


# ---------------------------------------------------------------------------------------------
# Convection-diffusion (Eq. 3)
# ---------------------------------------------------------------------------------------------
def test_cd_conserves_mass_exactly():
    cfg = cfg_small(grid=(5, 4, 6), ns=3, phi_p=0.4)
    shp = (3, 6, 4, 5)
    phi = 0.2 + 0.1 * inputs.uniform01(61, int(np.prod(shp))).reshape(shp)
    mu = inputs.random_field(shp, seed=62)
    u = 0.05 * inputs.random_field((3,) + shp[1:], seed=63)
    m0 = phi.reshape(3, -1).sum(1)
    out = oracle.cd_step(cfg, phi, mu, u, m0)
    assert np.abs(out.reshape(3, -1).sum(1) - m0).max() < 1e-12


def test_lax_wendroff_amplification_closed_form():
    """M = 0 leaves pure two-step Lax-Wendroff: G = 1 - i C sin(t) - C^2 (1 - cos t)."""
    L = 16
    cfg = cfg_small(grid=(L, 3, 2))
    cfg["M"] = 0.0
    C = 0.3
    th = 2 * np.pi * 3 / L
    z, y, x = np.meshgrid(np.arange(2), np.arange(3), np.arange(L), indexing="ij")
    eps = 1e-3
    phi = np.stack([0.5 + eps * np.cos(th * x), 0.5 - eps * np.cos(th * x)])
    u = np.zeros((3, 2, 3, L)); u[0] = C
    out = oracle.cd_step(cfg, phi, np.zeros_like(phi), u, phi.reshape(2, -1).sum(1))
    G = 1 - 1j * C * np.sin(th) - C * C * (1 - np.cos(th))
    ref = 0.5 + eps * np.real(G * np.exp(1j * th * x))
    assert np.abs(out[0] - ref).max() < 1e-15


def test_uniform_state_with_uniform_velocity_is_steady():
    cfg = cfg_small(grid=(4, 5, 3))
    phi = np.stack([np.full((3, 5, 4), 0.4), np.full((3, 5, 4), 0.6)])
    u = np.zeros((3, 3, 5, 4)); u[0], u[1], u[2] = 0.05, -0.02, 0.01
    out = oracle.cd_step(cfg, phi, np.full_like(phi, 0.3), u, phi.reshape(2, -1).sum(1))
    assert np.abs(out - phi).max() < 1e-15


# ---------------------------------------------------------------------------------------------
# Whole step: growth of small Fourier modes (linearised, RPA) in diffusion-only mode
# ---------------------------------------------------------------------------------------------
def rpa_amplification(cfg, kvec):
    """Closed-form 2x2 amplification of one step for a Fourier mode about the uniform melt."""
    N, nA = cfg["N"], cfg["nA"]
    s_hat = symbol(cfg["a"], kvec)
    types = [0] * nA + [1] * (N - nA)
    S = np.zeros((2, 2))
    for s in range(N):
        for t in range(N):
            S[types[s], types[t]] += s_hat ** abs(s - t)
    S *= cfg["phi_p"] / N
    chi = np.zeros((2, 2)); chi[0, 1] = chi[1, 0] = cfg["chi"][(0, 1)]
    kap = cfg["kappa"]
    ones = np.ones((2, 2))
    Mmu = np.linalg.inv(S) + s_hat * chi + kap * ones            # d mu / d phi
    phib = cfg["phi_p"] * np.array([nA / N, 1 - nA / N])
    Phi = np.diag(phib)
    k2 = sum(2 - 2 * np.cos(k) for k in kvec)
    dt, M = cfg["dt"], cfg["M"]
    c = 0.5 * dt * M
    H = np.diag(1 / phib) + kap * ones
    B = np.eye(2) + 6 * c * Phi @ H
    Binv = np.linalg.inv(B)
    It = Binv @ (c * (6 - k2) * Phi @ H)
    P = sum(np.linalg.matrix_power(It, j) for j in range(cfg["cn_sweeps"]))
    r = -dt * M * k2 * Phi @ Mmu
    return np.eye(2) + P @ Binv @ r


@pytest.mark.parametrize("mode", [(1, 0, 0), (1, 1, 0), (2, 1, 1)])
def test_rpa_growth_of_small_modes(mode):
    grid = (8, 8, 8)
    cfg = inputs.melt(grid, 8, 0.5, 20.0, hydro=0, ncg_iters=60, dt=0.4)
    cfg["nA"] = 3
    k = [2 * np.pi * m / 8 for m in mode]
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    wave = np.cos(k[0] * x + k[1] * y + k[2] * z)
    amp = np.array([1e-6, -0.4e-6])
    phib = np.array([3 / 8, 5 / 8])
    phi = phib[:, None, None, None] + amp[:, None, None, None] * wave[None]
    # start the inversion from the linear-response potential so it converges fully
    U0 = np.zeros_like(phi)
    out = oracle.step(cfg, phi, U0, None, phi.reshape(2, -1).sum(1))
    assert out["info"][-1] < 1e-14
    new = out["phi"] - phib[:, None, None, None]
    meas = (new * wave[None]).reshape(2, -1).sum(1) / (wave * wave).sum()
    A = rpa_amplification(cfg, k)
    assert np.abs(meas - A @ amp).max() < 1e-5 * np.abs(amp).max()


# ---------------------------------------------------------------------------------------------
# Free energy (Eq. 1) and order parameters (Fig. 1, Fig. 3)
# ---------------------------------------------------------------------------------------------
def test_free_energy_uniform_closed_form():
    cfg = cfg_small(grid=(3, 3, 3), chi=0.8)
    phi = np.stack([np.full((3, 3, 3), 0.5), np.full((3, 3, 3), 0.5)])
    assert abs(oracle.free_energy(cfg, np.zeros_like(phi), phi) - 0.8 * 0.25) < 1e-15


def test_free_energy_derivative_is_chemical_potential():
    """dF/dphi_I(r) = mu_I(r) (Eq. 4 is the functional derivative of Eq. 1), checked with a
    mass-conserving finite difference and fully converged potentials."""
    cfg = cfg_small(grid=(3, 2, 3), N=4, nA=2, chi=0.7, ncg_iters=200)
    shp = (2, 3, 2, 3)
    phi = 0.5 + 0.05 * inputs.random_field(shp, seed=71)
    phi[1] = 1.0 - phi[0] + 0.01 * inputs.random_field(shp[1:], seed=72)
    # block masses must equal those of the chains (V phi_p n_A / N each) for a solution to exist
    phi[0] *= 9.0 / phi[0].sum()
    phi[1] *= 9.0 / phi[1].sum()

    def F(ph):
        U, phim, info = oracle.ncg(cfg, ph, np.zeros_like(ph))
        assert info[-1] < 1e-12
        return oracle.free_energy(cfg, U, ph) * ph[0].size, U

    _, U = F(phi)
    mu = oracle.mu(cfg, U, phi)
    h = 1e-5
    i, j = (0, 1, 0, 2), (0, 2, 1, 0)
    pp = phi.copy(); pp[i] += h; pp[j] -= h
    pm = phi.copy(); pm[i] -= h; pm[j] += h
    fd = (F(pp)[0] - F(pm)[0]) / (2 * h)
    assert abs(fd - (mu[i] - mu[j])) < 1e-7


def test_order_parameters_closed_form():
    cfg = cfg_small(grid=(4, 1, 1), ns=3, phi_p=0.5)
    phi = np.zeros((3, 1, 1, 4))
    phi[0, 0, 0] = [0.1, 0.3, 0.1, 0.3]
    phi[1, 0, 0] = [0.2, 0.2, 0.4, 0.4]
    phi[2] = 1 - phi[0] - phi[1]
    dA = np.array([-0.1, 0.1, -0.1, 0.1]); dB = np.array([-0.1, -0.1, 0.1, 0.1])
    S = np.sqrt((dA ** 2 + dB ** 2 + (dA + dB) ** 2).sum() / 4)
    assert abs(oracle.order_parameter(cfg, phi) - S) < 1e-15
    assert abs(oracle.segregation(cfg, phi) - np.abs(dA + dB).mean()) < 1e-15


def test_mrt_forcing_second_moment_closed_form():
    """On one site (streaming maps it onto itself) the post-collision momentum flux is
    rho u u + rho/3 I + gamma_s dev(Pi_neq) + gamma_b tr(Pi_neq)/3 I + Sigma (Eq. 13-14), with u the
    half-force velocity of Eq. 9, Pi_neq the non-equilibrium second moment and Sigma of Eq. 14."""
    ts, tb = 0.7, 1.6
    gs, gb = 1 - 1 / ts, 1 - 1 / tb
    cfg = lb_cfg((1, 1, 1), ts, tb)
    _, w, _, c = oracle.lb_basis()
    rho, u0 = 1.03, np.array([0.02, -0.03, 0.01])
    n = oracle.lb_equilibrium(rho, u0) + 1e-3 * inputs.random_field((19,), seed=81) * w
    rho = n.sum()
    f = np.array([2e-3, 1e-3, -3e-3])
    out, uo = oracle.lb_step(cfg, n.reshape(19, 1, 1, 1), f.reshape(3, 1, 1, 1))
    cf = c.astype(float)
    u = (n @ cf + 0.5 * f) / rho
    assert np.abs(uo[:, 0, 0, 0] - u).max() < 1e-16
    Pi = np.einsum("i,ia,ib->ab", n, cf, cf)
    Pieq = rho * np.outer(u, u) + rho / 3 * np.eye(3)
    Pn = Pi - Pieq
    dev = Pn - np.trace(Pn) / 3 * np.eye(3)
    uf = u @ f
    Sig = 0.5 * (1 + gs) * (np.outer(u, f) + np.outer(f, u) - 2 / 3 * uf * np.eye(3)) + (1 + gb) / 3 * uf * np.eye(3)
    expect = Pieq + gs * dev + gb * np.trace(Pn) / 3 * np.eye(3) + Sig
    got = np.einsum("i,ia,ib->ab", out[:, 0, 0, 0], cf, cf)
    assert np.abs(got - expect).max() < 1e-15
    assert abs(out.sum() - rho) < 1e-15
    assert np.abs(out[:, 0, 0, 0] @ cf - (n @ cf + f)).max() < 1e-16


def test_uniform_chemical_potential_without_flow_is_stationary():
    """Nonuniform compositions at uniform mu feel no diffusive flux (Eq. 3 with u = 0)."""
    cfg = cfg_small(grid=(5, 4, 3), ns=3, phi_p=0.4)
    shp = (3, 3, 4, 5)
    phi = 0.2 + 0.15 * inputs.uniform01(91, int(np.prod(shp))).reshape(shp)
    mu = np.stack([np.full(shp[1:], v) for v in (0.3, -1.2, 0.7)])
    out = oracle.cd_step(cfg, phi, mu, None, phi.reshape(3, -1).sum(1))
    assert np.abs(out - phi).max() < 1e-15


def test_converged_crank_nicolson_conserves_mass_by_itself():
    """The Jacobi sweeps converge to the flux-form Crank-Nicolson solution, which conserves each
    species exactly (no mass shift applied here); two sweeps do not, which is why the step
    applies the shift."""
    shp = (2, 3, 4, 5)
    phi = 0.35 + 0.3 * inputs.uniform01(95, int(np.prod(shp))).reshape(shp)
    mu = 0.5 * inputs.random_field(shp, seed=96)
    m0 = phi.reshape(2, -1).sum(1)
    drift = {}
    for K in (2, 400):
        cfg = cfg_small(grid=(5, 4, 3), cn_sweeps=K)
        cfg["dt"] = 0.05
        out = oracle.cd_step(cfg, phi, mu, None, None)
        drift[K] = np.abs(out.reshape(2, -1).sum(1) - m0).max()
    assert drift[400] < 1e-13
    assert drift[2] > 1e-6


# ---------------------------------------------------------------------------------------------
# Learned-predictor network reference (circular 5^3 convolutions)
# ---------------------------------------------------------------------------------------------
def test_conv3d_equals_fft_correlation():
    grid = (6, 5, 7)
    nx, ny, nz = grid
    W = inputs.random_field((3, 2, 125), seed=101)
    b = inputs.random_field((3,), seed=102)
    x = inputs.random_field((2, 2, nz, ny, nx), seed=103)
    out = oracle.conv3d(grid, 2, W, b, x)
    # correlation theorem: out[co] = b + sum_ci ifft(fft(x_ci) * conj(fft(kernel_co_ci)))
    for n in range(2):
        for co in range(3):
            acc = np.full((nz, ny, nx), b[co])
            for ci in range(2):
                k = np.zeros((nz, ny, nx))
                for o in range(125):
                    oz, oy, ox = o // 25 - 2, (o // 5) % 5 - 2, o % 5 - 2
                    k[oz % nz, oy % ny, ox % nx] += W[co, ci, o]
                acc += np.real(np.fft.ifftn(np.fft.fftn(x[n, ci]) * np.conj(np.fft.fftn(k))))
            assert np.abs(out[n, co] - acc).max() < 1e-12


def test_conv3d_backward_finite_differences():
    grid = (5, 4, 6)
    nx, ny, nz = grid
    W = inputs.random_field((2, 3, 125), seed=111)
    b = inputs.random_field((2,), seed=112)
    x = inputs.random_field((1, 3, nz, ny, nx), seed=113)
    dout = inputs.random_field((1, 2, nz, ny, nx), seed=114)
    dW, db, din = oracle.conv3d_bwd(grid, 1, W, x, dout)
    f = lambda W_, b_, x_: float((oracle.conv3d(grid, 1, W_, b_, x_) * dout).sum())
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 62), (0, 1, 124)]:
        Wp = W.copy(); Wp[idx] += h
        Wm = W.copy(); Wm[idx] -= h
        assert abs((f(Wp, b, x) - f(Wm, b, x)) / (2 * h) - dW[idx]) < 1e-7 * max(1.0, abs(dW[idx]))
    bp = b.copy(); bp[1] += h
    bm = b.copy(); bm[1] -= h
    assert abs((f(W, bp, x) - f(W, bm, x)) / (2 * h) - db[1]) < 1e-7
    for idx in [(0, 0, 0, 0, 0), (0, 2, 5, 3, 4), (0, 1, 2, 1, 3)]:
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        assert abs((f(W, b, xp) - f(W, b, xm)) / (2 * h) - din[idx]) < 1e-7 * max(1.0, abs(din[idx]))


def test_net_gradient_finite_differences():
    """Whole-network gradient (mean removal, tanh layers) against central differences (1e-6 rel)."""
    grid = (4, 4, 4)
    rng = [inputs.random_field(s, seed=120 + i, scale=0.3) for i, s in
           enumerate([(4, 2, 125), (4,), (4, 4, 125), (4,), (2, 4, 125), (2,)])]
    params = [[rng[0], rng[1]], [rng[2], rng[3]], [rng[4], rng[5]]]
    U = inputs.random_field((2, 2, 4, 4, 4), seed=130, scale=0.5)
    tgt = 0.5 + 0.05 * inputs.random_field((2, 2, 4, 4, 4), seed=131)
    phibar = [0.5, 0.5]
    loss, grads = oracle.net_loss_grad(grid, params, U, tgt, phibar)
    h = 1e-6
    for (li, pi, idx) in [(0, 0, (1, 0, 17)), (1, 0, (2, 3, 99)), (2, 0, (1, 2, 60)), (0, 1, (3,)), (2, 1, (0,))]:
        P = [[a.copy(), b_.copy()] for a, b_ in params]
        P[li][pi][idx] += h
        lp = oracle.net_loss_grad(grid, P, U, tgt, phibar)[0]
        P[li][pi][idx] -= 2 * h
        lm = oracle.net_loss_grad(grid, P, U, tgt, phibar)[0]
        fd = (lp - lm) / (2 * h)
        g = grads[li][pi][idx]
        assert abs(fd - g) <= 1e-6 * max(abs(g), 1e-3 * abs(loss))


# ---------------------------------------------------------------------------------------------
# Thermal noise (Eq. 5, Eq. 13): the counter-based generator and the two noise terms
# ---------------------------------------------------------------------------------------------
def test_philox_known_answers():
    """The oracle's Philox4x32-10 reproduces the generator's published known-answer vectors."""
    kat = json.load(open(os.path.join(GOLDEN, "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        out = oracle.philox4x32([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert out == [int(x, 16) for x in v["out"]]


def test_normals_are_standard():
    """Box-Muller normals of distinct counters: mean 0, variance 1, kurtosis 3, pairs uncorrelated."""
    n = np.array([oracle.normals4(12345, site, 7, 3) for site in range(40000)])
    x = n.ravel()
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1.0) < 0.02
    assert abs((x ** 4).mean() / x.var() ** 2 - 3.0) < 0.08
    assert abs(np.corrcoef(n[:, 0], n[:, 1])[0, 1]) < 0.02
    assert abs(np.corrcoef(n[:, 0], n[:, 2])[0, 1]) < 0.02
    # different streams and steps give different numbers
    assert not np.allclose(oracle.normals4(1, 5, 0, 1), oracle.normals4(1, 5, 0, 2))
    assert not np.allclose(oracle.normals4(1, 5, 0, 1), oracle.normals4(1, 5, 1, 1))


def test_cd_noise_fluctuation_dissipation():
    """Composition noise of Eq. 5 as a random face flux: every species' total is kept exactly;
    for a uniform phi the increment has variance 12 M phi dt / Omega (six faces of variance
    2 M phi dt / Omega each) and neighbours along an axis share one face (covariance -1/6 of it)."""
    cfg = dict(cfg_small(grid=(24, 24, 24), N=4, nA=2), omega=100.0, noise_seed=99, noise_step=4)
    phi = np.stack([np.full((24, 24, 24), 0.3), np.full((24, 24, 24), 0.7)])
    dn = oracle.cd_noise(cfg, phi)
    assert np.abs(dn.reshape(2, -1).sum(1)).max() < 1e-12
    M, dt, om = cfg["M"], cfg["dt"], cfg["omega"]
    for I, ph in enumerate((0.3, 0.7)):
        var = 12 * M * ph * dt / om
        assert abs(dn[I].var() / var - 1.0) < 0.04
        for ax in range(3):
            cov = (dn[I] * np.roll(dn[I], -1, axis=ax)).mean()
            assert abs(cov / var + 1.0 / 6.0) < 0.03
    # species are independent, and a field-dependent amplitude follows phi_face
    assert abs(np.corrcoef(dn[0].ravel(), dn[1].ravel())[0, 1]) < 0.03
    phi2 = phi.copy()
    phi2[0] = 0.0
    assert np.abs(oracle.cd_noise(cfg, phi2)[0]).max() == 0.0


def test_lb_noise_conserves_and_has_the_mode_variances():
    """Fluctuating collision (Eq. 13): from rest, one step conserves mass and momentum at every
    site, and each non-conserved mode k = 4..18 of the post-collision populations has variance
    phi_k^2 = rho kT b_k (1 - gamma_k^2) / c_s^2 with kT = dt^2 / Omega."""
    g = (20, 20, 20)
    cfg = dict(cfg_small(grid=g, N=4, nA=2, tau_s=0.9, tau_b=1.3), omega=50.0, lb_noise=1,
               noise_seed=7, noise_step=2)
    e, w, b, c = oracle.lb_basis()
    n0 = np.broadcast_to(w[:, None, None, None], (19,) + g[::-1]).copy()
    out, _ = oracle.lb_step(cfg, n0)
    # undo the streaming: post-collision populations at each site
    post = np.stack([np.roll(out[i], shift=(-c[i][2], -c[i][1], -c[i][0]), axis=(0, 1, 2)) for i in range(19)])
    m = np.tensordot(e, post - w[:, None, None, None], axes=(1, 0))
    assert np.abs(m[0]).max() < 1e-14 and np.abs(m[1:4]).max() < 1e-14
    kT = cfg["dt"] ** 2 / cfg["omega"]
    gs, gb = 1 - 1 / cfg["tau_s"], 1 - 1 / cfg["tau_b"]
    gam = [gb] + [gs] * 5 + [0.0] * 9
    for k in range(4, 19):
        expect = kT * b[k] * (1 - gam[k - 4] ** 2) * 3.0
        assert abs(m[k].var() / expect - 1.0) < 0.06, k
        assert abs(m[k].mean()) < 4 * np.sqrt(expect / m[k].size)


# ---------------------------------------------------------------------------------------------
# Minkowski functionals of a thresholded field (Sec. 3; Michielsen-De Raedt voxel counting)
# ---------------------------------------------------------------------------------------------
def _body(shape, cells):
    g = np.zeros(shape)
    for c in cells:
        g[c] = 1.0
    return g


def test_minkowski_closed_forms():
    """Volume, area, mean-breadth term and Euler characteristic of bodies whose values are known:
    a unit cube (1, 6, 3, 1), two disjoint cubes (additive), a 3^3 cube with a central cavity
    (a hollow ball: chi = 2; area 54 outside + 6 inside), a ring (solid torus: chi = 0), a rod
    closing on itself through the periodic box (chi = 0), the filled box (a 3-torus: 0, no
    surface), cubes touching at a corner (one connected closed body: chi = 1)."""
    cube = oracle.minkowski(_body((8, 8, 8), [(3, 3, 3)]), 0.5)
    assert cube == {"V": 1, "S": 6, "B2": 3, "chi": 1}
    two = oracle.minkowski(_body((8, 8, 8), [(1, 1, 1), (5, 5, 5)]), 0.5)
    assert two == {"V": 2, "S": 12, "B2": 6, "chi": 2}
    g = np.zeros((9, 9, 9))
    g[2:5, 2:5, 2:5] = 1.0
    g[3, 3, 3] = 0.0
    shell = oracle.minkowski(g, 0.5)
    assert shell["V"] == 26 and shell["S"] == 60 and shell["chi"] == 2
    ring = np.zeros((8, 8, 8))
    ring[3, 2:5, 2:5] = 1.0
    ring[3, 3, 3] = 0.0
    assert oracle.minkowski(ring, 0.5)["chi"] == 0
    rod = np.zeros((8, 8, 8))
    rod[:, 3, 3] = 1.0
    assert oracle.minkowski(rod, 0.5) == {"V": 8, "S": 32, "B2": 8, "chi": 0}
    assert oracle.minkowski(np.ones((6, 6, 6)), 0.5) == {"V": 216, "S": 0, "B2": 0, "chi": 0}
    assert oracle.minkowski(_body((8, 8, 8), [(3, 3, 3), (4, 4, 4)]), 0.5)["chi"] == 1


def test_minkowski_invariances():
    """A random body: the counts do not change under periodic translation or under axis
    permutations, the threshold is strict, and a scaled copy scales V by 8 and S by 4."""
    rng = np.random.default_rng(5)
    f = rng.random((10, 12, 14))
    c0 = oracle.minkowski_counts(f, 0.6)
    assert oracle.minkowski_counts(np.roll(f, (3, -5, 7), axis=(0, 1, 2)), 0.6) == c0
    assert oracle.minkowski_counts(np.ascontiguousarray(f.transpose(2, 0, 1)), 0.6) == c0
    assert oracle.minkowski_counts(np.full((4, 4, 4), 0.6), 0.6)[0] == 0
    b = (rng.random((5, 6, 7)) > 0.7).astype(float)
    big = np.kron(b, np.ones((2, 2, 2)))
    m1, m2 = oracle.minkowski(b, 0.5), oracle.minkowski(big, 0.5)
    assert m2["V"] == 8 * m1["V"] and m2["S"] == 4 * m1["S"] and m2["chi"] == m1["chi"]


def test_trapped_solvent_closed_forms():
    """Trapped solvent: the solvent inside closed B shells, as a fraction of all solvent.  One
    hollow cube traps exactly its cavity; two shells trap both cavities; an open cup, a slab and
    an empty box trap nothing; the result does not depend on where the box is cut."""
    shape = (12, 12, 12)
    phiS = 0.5 + 0.1 * inputs.uniform01(3, 12 ** 3).reshape(shape)
    B = np.zeros(shape)
    B[2:7, 2:7, 2:7] = 1.0
    B[3:6, 3:6, 3:6] = 0.0        # cavity of 27 sites
    f, n = oracle.trapped_solvent(B, phiS)
    cav = np.zeros(shape, bool)
    cav[3:6, 3:6, 3:6] = True
    assert n == 2 and abs(f - phiS[cav].sum() / phiS.sum()) < 1e-14
    B2 = B.copy()
    B2[8:11, 8:11, 8:11] = 1.0
    B2[9, 9, 9] = 0.0              # a second shell, cavity of one site
    cav2 = cav.copy()
    cav2[9, 9, 9] = True
    f2, n2 = oracle.trapped_solvent(B2, phiS)
    assert n2 == 3 and abs(f2 - phiS[cav2].sum() / phiS.sum()) < 1e-14
    cup = B.copy()
    cup[6, 4, 4] = 0.0             # a hole in the lid: the cavity joins the bulk
    assert oracle.trapped_solvent(cup, phiS)[0] == 0.0
    slab = np.zeros(shape)
    slab[:, :, 5] = 1.0            # the complement stays connected through the periodic box
    assert oracle.trapped_solvent(slab, phiS) == (0.0, 1)
    assert oracle.trapped_solvent(np.zeros(shape), phiS) == (0.0, 1)
    sh = (4, -3, 5)
    fr, nr = oracle.trapped_solvent(np.roll(B2, sh, axis=(0, 1, 2)), np.roll(phiS, sh, axis=(0, 1, 2)))
    assert nr == n2 and abs(fr - f2) < 1e-14


def test_trapped_solvent_against_library_labelling():
    """The oracle's breadth-first components against an independent labelling: scipy's
    face-connected labels of the complement in the open box, joined across the periodic faces by
    a union-find, on random fields at several thresholds (component count, largest component and
    the enclosed solvent fraction)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2024)
    for shape in [(9, 11, 13), (16, 8, 12)]:
        phiB = rng.random(shape)
        phiS = 0.2 + rng.random(shape)
        for th in (0.35, 0.5, 0.62):
            comp = phiB <= th
            lab, n = ndimage.label(comp, structure=ndimage.generate_binary_structure(3, 1))
            parent = list(range(n + 1))

            def find(a):
                while parent[a] != a:
                    parent[a] = parent[parent[a]]
                    a = parent[a]
                return a
            for ax in range(3):
                lo = np.take(lab, 0, axis=ax)
                hi = np.take(lab, shape[ax] - 1, axis=ax)
                for a, b in zip(lo.ravel(), hi.ravel()):
                    if a and b:
                        ra, rb = find(a), find(b)
                        if ra != rb:
                            parent[max(ra, rb)] = min(ra, rb)
            roots = np.array([find(a) if a else 0 for a in lab.ravel()]).reshape(shape)
            ids, sizes = np.unique(roots[roots > 0], return_counts=True)
            # the bulk: largest, ties to the component holding the smallest site index
            first = {i: np.flatnonzero(roots.ravel() == i)[0] for i in ids}
            bulk = min(ids, key=lambda i: (-sizes[list(ids).index(i)], first[i]))
            want = phiS[(roots > 0) & (roots != bulk)].sum() / phiS.sum()
            f, nc = oracle.trapped_solvent(phiB, phiS, th)
            assert nc == len(ids), (shape, th)
            assert abs(f - want) < 1e-13, (shape, th)


def test_minkowski_counts_against_enumeration():
    """The cube, face, edge and vertex counts of the body (the union of closed unit voxels of the
    periodic box) against a plain enumeration: every voxel contributes its 6 faces, 12 edges and 8
    corners, each named by its lattice position (wrapped), and the distinct ones are counted."""
    rng = np.random.default_rng(77)
    for shape, th in [((7, 9, 8), 0.55), ((6, 6, 10), 0.8), ((8, 5, 7), 0.3)]:
        f = rng.random(shape)
        nz, ny, nx = shape
        body = np.argwhere(f > th)
        faces, edges, verts = set(), set(), set()
        for z, y, x in body:
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        verts.add(((z + dz) % nz, (y + dy) % ny, (x + dx) % nx))
            # edges along x, y, z: the two other coordinates take both corner offsets
            for a in (0, 1):
                for c in (0, 1):
                    edges.add(("x", (z + a) % nz, (y + c) % ny, x % nx))
                    edges.add(("y", (z + a) % nz, y % ny, (x + c) % nx))
                    edges.add(("z", z % nz, (y + a) % ny, (x + c) % nx))
            for a in (0, 1):
                faces.add(("x", z, y, (x + a) % nx))
                faces.add(("y", z, (y + a) % ny, x))
                faces.add(("z", (z + a) % nz, y, x))
        want = (len(body), len(faces), len(edges), len(verts))
        got = oracle.minkowski_counts(f, th)
        assert tuple(got) == want, (shape, got, want)


# ---------------------------------------------------------------------------------------------
# Coupling of the two solvers (Sec. 2: the force of Eq. 8 drives the LB of Eq. 9-14, whose
# velocity advects the compositions in Eq. 3).  These pin the unit conversion between the
# Brownian time step dt and the LB step (force dt^2 f in lattice units, velocity u_lat = dt u
# handed to the convection step as a Courant number) with physics, not with the oracle's own
# formula: Newton's second law for a fluid starting from rest, the continuity equation, the
# gradient form of the linearised force, and the dissipation of the total energy.
# ---------------------------------------------------------------------------------------------
def _lb_energies(pop, dt):
    """Kinetic and compressional energy per site of the LB fluid in k_B T (rho0 = 1 m0/h^3, so
    m0 h^2/tau^2 = k_B T): (1/2) j^2/rho in physical velocity j/(rho dt), and c_s^2 drho^2/2
    with the physical sound speed c_s^2 = h^2/(3 dt^2)."""
    _, _, _, c = oracle.lb_basis()
    rho = pop.sum(0)
    j = np.einsum("izyx,ia->azyx", pop, c.astype(float))
    return (0.5 * (j * j).sum(0) / rho).mean() / dt ** 2, ((rho - 1.0) ** 2).mean() / (6.0 * dt * dt)


def _spectral_divergence(flux):
    """div of flux [I][3][nz][ny][nx] (components x, y, z) by FFT: the continuum operator."""
    out = np.zeros((flux.shape[0],) + flux.shape[2:])
    for a, ax in ((0, 3), (1, 2), (2, 1)):
        n = flux.shape[ax + 1]
        kk = (2j * np.pi * np.fft.fftfreq(n)).reshape([n if d == ax else 1 for d in range(4)])
        out += np.real(np.fft.ifftn(np.fft.fftn(flux[:, a], axes=(1, 2, 3)) * kk, axes=(1, 2, 3)))
    return out


@pytest.mark.parametrize("dt", [0.1, 0.05])
def test_hydro_first_step_from_rest_obeys_newton_and_advects(dt):
    """A fluid at rest under the body force f of Eq. 8 moves during the first step with the mean
    velocity dt f/(2 rho0) (Newton; Eq. 9's half-force velocity is that mean), so the Courant
    number the step reports is dt^2 f/(2 rho0), and with M = 0 the compositions change only by
    the continuity equation, -dt div(phi u) (Eq. 3), here compared with the continuum
    divergence (tolerance: the O((k h)^2) difference of the lattice fluxes, about 2.5% for these
    wavelengths).  A force scaled by dt instead of dt^2, or a velocity handed to the convection
    step in other units than the Courant number, is off by a factor 1/dt."""
    grid = (32, 32, 2)
    cfg = inputs.melt(grid, 8, 0.5, 12.0, hydro=1, ncg_iters=40, dt=dt)
    cfg["M"] = 0.0
    z, y, x = np.meshgrid(np.arange(2), np.arange(32), np.arange(32), indexing="ij")
    k = 2 * np.pi / 32
    w1, w2 = np.cos(k * x), np.cos(k * (x + 2 * y) + 0.3)
    phi = np.stack([0.5 + 0.02 * (w1 + 0.5 * w2), 0.5 - 0.02 * (w1 + 0.5 * w2) + 0.01 * w2])
    out = oracle.step(cfg, phi, np.zeros_like(phi), None, phi.reshape(2, -1).sum(1))
    assert out["info"][-1] < 1e-8
    f = oracle.force(cfg, phi, out["mu"])
    ubar = dt * f / (2.0 * cfg["rho0"])                      # physical mean velocity, h/tau
    assert np.abs(out["ulat"] - dt * ubar).max() <= 1e-12 * np.abs(dt * ubar).max()
    dphi = out["phi"] - phi
    cont = -dt * _spectral_divergence(phi[:, None] * ubar[None])
    assert np.abs(dphi - cont).max() <= 0.05 * np.abs(cont).max()
    assert np.abs(cont).max() > 1e-3 * dt * dt          # the advection is resolved


def _helmholtz(u):
    """Longitudinal and transverse parts of a periodic vector field [3][nz][ny][nx]."""
    nz, ny, nx = u.shape[1:]
    kz, ky, kx = np.meshgrid(np.fft.fftfreq(nz), np.fft.fftfreq(ny), np.fft.fftfreq(nx), indexing="ij")
    K = np.stack([kx, ky, kz])
    k2 = (K * K).sum(0)
    k2[0, 0, 0] = 1.0
    Uk = np.fft.fftn(u, axes=(1, 2, 3))
    UL = K * (K * Uk).sum(0) / k2
    return np.real(np.fft.ifftn(UL, axes=(1, 2, 3))), np.real(np.fft.ifftn(Uk - UL, axes=(1, 2, 3)))


def test_hydro_transverse_velocity_is_second_order():
    """Linearised about the uniform melt, f = -sum_I phi_I grad mu_I = -grad(sum_I phibar_I dmu_I)
    + O(delta^2) is a gradient (Eq. 8), so it drives only the longitudinal (sound) part of the LB
    velocity: over a few coupled steps the longitudinal velocity grows linearly with the amplitude
    delta of a two-mode perturbation and the transverse one quadratically (the modes have
    different |k|, so the second-order force has a curl).  A force whose components pair with the
    wrong derivatives, or any non-gradient linear term, makes the transverse part linear."""
    L = 16
    grid = (L, L, 2)
    z, y, x = np.meshgrid(np.arange(2), np.arange(L), np.arange(L), indexing="ij")
    k = 2 * np.pi / L
    w1, w2 = np.cos(k * x), np.cos(2 * k * y + 0.4)
    parts = {}
    for amp in (1e-3, 2e-3):
        cfg = inputs.melt(grid, 8, 0.5, 12.0, hydro=1, ncg_iters=40, dt=0.1)
        phi = np.stack([0.5 + amp * (w1 + w2), 0.5 - amp * w1 + 0.5 * amp * w2])
        U, pop, m0 = np.zeros_like(phi), None, phi.reshape(2, -1).sum(1)
        for _ in range(6):
            o = oracle.step(cfg, phi, U, pop, m0)
            phi, U, pop = o["phi"], o["U"], o["pop"]
        uL, uT = _helmholtz(o["ulat"])
        parts[amp] = (np.abs(uL).max(), np.abs(uT).max())
    (l1, t1), (l2, t2) = parts[1e-3], parts[2e-3]
    assert abs(l2 / l1 - 2.0) < 2e-3
    assert abs(t2 / t1 - 4.0) < 2e-2
    assert t1 < 1e-3 * l1


def test_diffusion_only_free_energy_is_non_increasing():
    """Without flow, Eq. 3 is a gradient flow of the free energy of Eq. 1 (dF/dt = -int M phi
    |grad mu|^2 <= 0): F(t) of a quenched melt must not increase from step to step at dt = 0.1."""
    cfg = inputs.melt((12, 12, 12), 8, 0.5, 16.0, noise=0.05, seed=7, dt=0.1, hydro=0, ncg_iters=30)
    phi = inputs.initial_fields(cfg)
    U, m0 = np.zeros_like(phi), phi.reshape(2, -1).sum(1)
    F = []
    for _ in range(30):
        o = oracle.step(cfg, phi, U, None, m0)
        F.append(oracle.free_energy(cfg, o["U"], phi))      # F of phi^n at its potentials U^n
        phi, U = o["phi"], o["U"]
    assert np.diff(F).max() < 0.0
    assert F[0] - F[-1] > 1e-3


def test_hydro_total_energy_is_non_increasing():
    """With the LB coupled, the free energy released by advection is the work the force of Eq. 8
    does on the fluid, so F + (kinetic + compressional energy of the LB fluid) is what decreases
    (diffusive and viscous dissipation).  From a quench with a compressive perturbation, where
    the flow carries energy comparable to the changes of F, the total must not increase at
    dt = 0.1.  A force in lattice units too large by 1/dt pumps energy in and fails at once."""
    grid = (16, 16, 16)
    cfg = inputs.melt(grid, 8, 0.5, 16.0, noise=0.03, seed=5, dt=0.1, hydro=1, ncg_iters=30)
    phi = inputs.initial_fields(cfg)
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    phi[1] += 0.03 * np.cos(2 * np.pi * x / 16) * np.cos(2 * np.pi * y / 16)
    U, pop, m0 = np.zeros_like(phi), None, phi.reshape(2, -1).sum(1)
    E, kin = [], []
    for _ in range(40):
        o = oracle.step(cfg, phi, U, pop, m0)
        ke, pe = _lb_energies(pop, cfg["dt"]) if pop is not None else (0.0, 0.0)
        E.append(oracle.free_energy(cfg, o["U"], phi) + ke + pe)
        kin.append(ke + pe)
        phi, U, pop = o["phi"], o["U"], o["pop"]
    assert np.diff(E).max() < 0.0
    assert max(kin) > 1e-5          # the flow matters in this run


# ---------------------------------------------------------------------------------------------
# Starting point of the inversion (the paper does not give it): the previous step's potentials
# or their linear extrapolation in time.  Neither changes what the inversion converges to; the
# extrapolation makes the starting residual second order in the time step instead of first.
# ---------------------------------------------------------------------------------------------
def _run_start_residuals(cfg, steps, extrap):
    phi = inputs.initial_fields(cfg)
    U, Up, m0 = np.zeros_like(phi), None, phi.reshape(2, -1).sum(1)
    c = dict(cfg, warm_extrap=1 if extrap else 0)
    res, out = [], []
    for k in range(steps):
        # history: the incoming U of the previous step, once that step started from an inversion's
        # result (from the third step on; the first starts from the cold U = 0)
        st = oracle.step(c, phi, U, None, m0, Uprev=Up if k >= 2 else None)
        res.append(st["info"][1])                 # max|phi* - phi[U]| where the inversion starts
        phi, U, Up = st["phi"], st["U"], st["Uprev"]
        out.append(phi)
    return np.array(res), out


def test_extrapolated_start_converges_to_the_same_state():
    cfg = inputs.melt((10, 10, 10), 8, 0.5, 12.0, noise=0.05, seed=9, dt=0.02, hydro=0, ncg_iters=200)
    cfg["ncg_tol"] = 1e-12
    r0, plain = _run_start_residuals(cfg, 8, False)
    r1, extr = _run_start_residuals(cfg, 8, True)
    for a, b in zip(plain, extr):
        assert np.abs(a - b).max() < 1e-10
    assert (r1[:2] == r0[:2]).all()                # no history yet
    assert (r1[3:] < 0.3 * r0[3:]).all()


def test_extrapolated_start_residual_is_second_order_in_dt():
    """Without extrapolation the starting residual is the composition change of one step, O(dt);
    with it, O(dt^2): halving dt halves the first and quarters the second (after the quench
    transient, at the same physical time)."""
    res = {}
    for dt in (0.02, 0.01):
        n = int(round(0.2 / dt))
        cfg = inputs.melt((10, 10, 10), 8, 0.5, 12.0, noise=0.05, seed=9, dt=dt, hydro=0, ncg_iters=200)
        cfg["ncg_tol"] = 1e-12
        res[dt] = (_run_start_residuals(cfg, n, False)[0][-1], _run_start_residuals(cfg, n, True)[0][-1])
    plain = res[0.02][0] / res[0.01][0]
    extr = res[0.02][1] / res[0.01][1]
    assert 1.7 < plain < 2.3
    assert 3.3 < extr < 4.9
