"""FP64 CPU oracle for the hybrid LB / dynamic SCF time step (arXiv:1204.2088).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The product path (the CUDA library and its
binding) never imports, links or executes anything here, and nothing here imports the
product.  The arithmetic lives in ``oracle.c`` (plain C, FP64); this module only marshals
numpy arrays through ctypes.

Parity status of each function (what pins it is in ``tests/test_oracle_pins.py``):
  sigma, densities, objective, ncg, mu, force, lb_step, cd_step, step, free_energy,
  order_parameter, segregation: pinned.  The coupling inside ``step`` (the force of Eq. 8 in
  lattice units, dt^2 f, and the LB velocity handed to the convection step as the Courant number
  dt u) is pinned by Newton's law for a fluid starting from rest with the continuity equation,
  by the gradient form of the linearised force (transverse velocity of second order) and by the
  decrease of F, and of F plus the LB fluid's kinetic and compressional energy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, FP64, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("ns", ctypes.c_int32), ("N", ctypes.c_int32), ("nA", ctypes.c_int32),
        ("phi_p", ctypes.c_double), ("chi", ctypes.c_double * 9), ("kappa", ctypes.c_double),
        ("a", ctypes.c_double), ("dt", ctypes.c_double), ("M", ctypes.c_double),
        ("tau_s", ctypes.c_double), ("tau_b", ctypes.c_double), ("rho0", ctypes.c_double),
        ("hydro", ctypes.c_int32), ("ncg_iters", ctypes.c_int32), ("cn_sweeps", ctypes.c_int32),
        ("phi_floor", ctypes.c_double), ("ncg_tol", ctypes.c_double),
        ("omega", ctypes.c_double), ("lb_noise", ctypes.c_int32), ("warm_extrap", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("step", ctypes.c_int64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(Params)
        sig = {
            "or_stencil_weights": (None, [ctypes.c_double, D]),
            "or_sigma": (None, [P, D, D]),
            "or_densities": (ctypes.c_double, [P, D, D, D, D]),
            "or_objective": (ctypes.c_double, [P, D, D]),
            "or_ncg": (ctypes.c_int, [P, D, D, D, D]),
            "or_philox4x32": (None, [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                     ctypes.POINTER(ctypes.c_uint32)]),
            "or_normals4": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, D]),
            "or_cd_noise": (None, [P, D, D]),
            "or_minkowski_counts": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_int64)]),
            "or_trapped_solvent": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, ctypes.c_double,
                                                     ctypes.POINTER(ctypes.c_int64)]),
            "or_mu": (None, [P, D, D, D]),
            "or_force": (None, [P, D, D, D]),
            "or_lb_basis": (None, [D, D, D, ctypes.POINTER(ctypes.c_int)]),
            "or_lb_equilibrium": (None, [ctypes.c_double, D, D]),
            "or_lb_step": (None, [P, D, D, D, D]),
            "or_cd_step": (None, [P, D, D, D, D, D]),
            "or_step": (None, [P, D, D, D, D, D, D, D, D, D]),
            "or_extrapolate": (None, [P, D, D]),
            "or_free_energy": (ctypes.c_double, [P, D, D]),
            "or_order_parameter": (ctypes.c_double, [P, D]),
            "or_segregation": (ctypes.c_double, [P, D]),
            "or_num_threads": (ctypes.c_int, []),
            "or_conv3d": (None, [ctypes.c_int] * 6 + [D, D, D, D]),
            "or_conv3d_bwd": (None, [ctypes.c_int] * 6 + [D, D, D, D, D, D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def make_params(cfg: dict) -> Params:
    """Build the oracle parameter struct from a plain configuration dictionary."""
    p = Params()
    p.nx, p.ny, p.nz = cfg["grid"]
    p.ns = cfg.get("ns", 2)
    p.N = cfg["N"]
    p.nA = cfg["nA"]
    p.phi_p = cfg.get("phi_p", 1.0)
    chi = np.zeros((3, 3))
    for (i, j), v in cfg.get("chi", {}).items():
        chi[i, j] = chi[j, i] = v
    for k in range(9):
        p.chi[k] = float(chi.flat[k])
    p.kappa = cfg.get("kappa", 10.0)
    p.a = cfg.get("a", 1.1543)
    p.dt = cfg.get("dt", 0.4)
    p.M = cfg.get("M", 1.0)
    p.tau_s = cfg.get("tau_s", 1.0)
    p.tau_b = cfg.get("tau_b", 1.0)
    p.rho0 = cfg.get("rho0", 1.0)
    p.hydro = cfg.get("hydro", 1)
    p.ncg_iters = cfg.get("ncg_iters", 4)
    p.cn_sweeps = cfg.get("cn_sweeps", 8)
    p.phi_floor = cfg.get("phi_floor", 1e-6)
    p.ncg_tol = cfg.get("ncg_tol", 0.0)
    p.omega = cfg.get("omega", 0.0)          # thermal noise (0: none)
    p.lb_noise = cfg.get("lb_noise", 0)
    p.seed = cfg.get("noise_seed", 0)
    p.warm_extrap = cfg.get("warm_extrap", 0)
    p.step = cfg.get("noise_step", 0)
    return p


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _shape(cfg):
    nx, ny, nz = cfg["grid"]
    return (nz, ny, nx)


def stencil_weights(a: float) -> np.ndarray:
    w = np.zeros(4)
    lib().or_stencil_weights(a, _ptr(w))
    return w


def sigma(cfg: dict, f: np.ndarray) -> np.ndarray:
    p = make_params(cfg)
    f = _f64(f)
    out = np.empty_like(f)
    lib().or_sigma(ctypes.byref(p), _ptr(f), _ptr(out))
    return out


def densities(cfg: dict, U: np.ndarray, want_stack: bool = False):
    """phi[U] (shape [ns, nz, ny, nx]), Q, <exp(-U_S)> and optionally G_0..G_N."""
    p = make_params(cfg)
    U = _f64(U)
    phi = np.empty_like(U)
    qs = ctypes.c_double(1.0)
    stack = None
    if want_stack:
        stack = np.empty((cfg["N"] + 1,) + _shape(cfg))
    Q = lib().or_densities(ctypes.byref(p), _ptr(U), _ptr(phi), ctypes.byref(qs),
                           _ptr(stack) if stack is not None else None)
    if want_stack:
        return phi, Q, qs.value, stack
    return phi, Q, qs.value


def objective(cfg: dict, U: np.ndarray, phi_target: np.ndarray) -> float:
    p = make_params(cfg)
    return lib().or_objective(ctypes.byref(p), _ptr(_f64(U)), _ptr(_f64(phi_target)))


def ncg(cfg: dict, phi_target: np.ndarray, U0: np.ndarray):
    """Fletcher-Reeves inversion: at most ncg_iters iterations, fewer once max|g| < ncg_tol
    (if ncg_tol > 0).  Returns (U, phi_model, info); ncg_run also gives the iterations run."""
    U, phim, info, _ = ncg_run(cfg, phi_target, U0)
    return U, phim, info


def ncg_run(cfg: dict, phi_target: np.ndarray, U0: np.ndarray):
    """As ncg, also returning the number of iterations run."""
    p = make_params(cfg)
    U = _f64(U0).copy()
    phim = np.empty_like(U)
    info = np.zeros(2 + 4 * max(cfg.get("ncg_iters", 4), 0))
    k = lib().or_ncg(ctypes.byref(p), _ptr(_f64(phi_target)), _ptr(U), _ptr(phim), _ptr(info))
    return U, phim, info, k


def philox4x32(ctr, key):
    """Philox4x32-10 of a counter (4 words) and key (2 words): 4 output words."""
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32(c, k, o)
    return list(o)


def normals4(seed: int, site: int, step: int, stream: int) -> np.ndarray:
    out = np.zeros(4)
    lib().or_normals4(seed, site, step, stream, _ptr(out))
    return out


def cd_noise(cfg: dict, phi: np.ndarray) -> np.ndarray:
    """The composition noise increment of one step (cfg: omega, noise_seed, noise_step)."""
    p = make_params(cfg)
    out = np.empty_like(_f64(phi))
    lib().or_cd_noise(ctypes.byref(p), _ptr(_f64(phi)), _ptr(out))
    return out


def minkowski_counts(field: np.ndarray, threshold: float):
    """(n_c, n_f, n_e, n_v) of the union of cubes where field > threshold; field [nz, ny, nx]."""
    f = _f64(field)
    nz, ny, nx = f.shape
    out = (ctypes.c_int64 * 4)()
    lib().or_minkowski_counts(nx, ny, nz, _ptr(f), threshold, out)
    return tuple(out)


def minkowski(field: np.ndarray, threshold: float) -> dict:
    """Volume, surface, 2 x integral mean curvature and Euler characteristic (voxel union)."""
    nc, nf, ne, nv = minkowski_counts(field, threshold)
    return {"V": nc, "S": -6 * nc + 2 * nf, "B2": 3 * nc - 2 * nf + ne, "chi": -nc + nf - ne + nv}


def trapped_solvent(phiB: np.ndarray, phiS: np.ndarray, threshold: float = 0.2):
    """(f_trap, number of components of the complement of {phi_B > threshold})."""
    b, s_ = _f64(phiB), _f64(phiS)
    nz, ny, nx = b.shape
    n = ctypes.c_int64()
    f = lib().or_trapped_solvent(nx, ny, nz, _ptr(b), _ptr(s_), threshold, ctypes.byref(n))
    return f, n.value


def mu(cfg: dict, U: np.ndarray, phi: np.ndarray) -> np.ndarray:
    p = make_params(cfg)
    out = np.empty_like(_f64(phi))
    lib().or_mu(ctypes.byref(p), _ptr(_f64(U)), _ptr(_f64(phi)), _ptr(out))
    return out


def force(cfg: dict, phi: np.ndarray, mu_: np.ndarray) -> np.ndarray:
    p = make_params(cfg)
    out = np.empty((3,) + _shape(cfg))
    lib().or_force(ctypes.byref(p), _ptr(_f64(phi)), _ptr(_f64(mu_)), _ptr(out))
    return out


def lb_basis():
    """(e[19,19], w[19], b[19], c[19,3]) of Table 1 with the D3Q19 velocities."""
    e = np.zeros((19, 19)); w = np.zeros(19); b = np.zeros(19)
    c = np.zeros((19, 3), dtype=np.intc)
    lib().or_lb_basis(_ptr(e), _ptr(w), _ptr(b), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e, w, b, c


def lb_equilibrium(rho: float, u) -> np.ndarray:
    out = np.zeros(19)
    lib().or_lb_equilibrium(float(rho), _ptr(_f64(u)), _ptr(out))
    return out


def lb_step(cfg: dict, n: np.ndarray, f_lat: np.ndarray | None = None):
    """One collide+stream step.  n: [19, nz, ny, nx] post-streaming populations."""
    p = make_params(cfg)
    n = _f64(n)
    out = np.empty_like(n)
    u = np.empty((3,) + _shape(cfg))
    lib().or_lb_step(ctypes.byref(p), _ptr(n), _ptr(_f64(f_lat)) if f_lat is not None else None,
                     _ptr(out), _ptr(u))
    return out, u


def cd_step(cfg: dict, phi: np.ndarray, mu_: np.ndarray, ulat: np.ndarray | None, mass0) -> np.ndarray:
    p = make_params(cfg)
    phi = _f64(phi)
    out = np.empty_like(phi)
    lib().or_cd_step(ctypes.byref(p), _ptr(phi), _ptr(_f64(mu_)),
                     _ptr(_f64(ulat)) if ulat is not None else None,
                     _ptr(_f64(mass0)) if mass0 is not None else None, _ptr(out))
    return out


def step(cfg: dict, phi: np.ndarray, U: np.ndarray, pop: np.ndarray | None, mass0, Uprev=None):
    """One coupled time step.  Returns a dict with the new state and the step outputs; "Uprev"
    holds a copy of the incoming U.  With cfg["warm_extrap"] and Uprev given (the incoming U of
    the previous step, itself the result of an inversion) the inversion starts from
    2 U - Uprev; without Uprev it starts from U."""
    p = make_params(cfg)
    U_in = _f64(U).copy()
    up = _f64(Uprev).copy() if (p.warm_extrap and Uprev is not None) else None
    phi = _f64(phi).copy()
    U = _f64(U).copy()
    shp = _shape(cfg)
    if pop is None:
        pop = np.zeros((19,) + shp)
        _, w, _, _ = lb_basis()
        pop += (cfg.get("rho0", 1.0) * w)[:, None, None, None]
    pop = _f64(pop).copy()
    mu_ = np.empty_like(phi)
    ulat = np.empty((3,) + shp)
    phim = np.empty_like(phi)
    info = np.zeros(2 + 4 * max(cfg.get("ncg_iters", 4), 0))
    lib().or_step(ctypes.byref(p), _ptr(phi), _ptr(U), _ptr(pop), _ptr(_f64(mass0)), _ptr(mu_),
                  _ptr(ulat), _ptr(phim), _ptr(info), _ptr(up) if up is not None else None)
    return {"phi": phi, "U": U, "pop": pop, "mu": mu_, "ulat": ulat, "phim": phim, "info": info, "Uprev": U_in}


def free_energy(cfg: dict, U: np.ndarray, phi: np.ndarray) -> float:
    p = make_params(cfg)
    return lib().or_free_energy(ctypes.byref(p), _ptr(_f64(U)), _ptr(_f64(phi)))


def order_parameter(cfg: dict, phi: np.ndarray) -> float:
    p = make_params(cfg)
    return lib().or_order_parameter(ctypes.byref(p), _ptr(_f64(phi)))


def segregation(cfg: dict, phi: np.ndarray) -> float:
    p = make_params(cfg)
    return lib().or_segregation(ctypes.byref(p), _ptr(_f64(phi)))


def num_threads() -> int:
    return lib().or_num_threads()


# ---------------------------------------------------------------------------------------------
# Learned predictor: FP64 reference of the 3-layer circular 5^3 convolution network
# (conv primitives in oracle.c, the composition below in numpy).
# ---------------------------------------------------------------------------------------------
NET_LAYERS = ((2, 32), (32, 32), (32, 2))


def conv3d(grid, batch, W, b, x):
    """x: [batch, cin, nz, ny, nx] -> [batch, cout, nz, ny, nx]."""
    nx, ny, nz = grid
    cout, cin = W.shape[0], W.shape[1]
    x = _f64(x)
    out = np.empty((batch, cout, nz, ny, nx))
    lib().or_conv3d(nx, ny, nz, batch, cin, cout, _ptr(_f64(W)), _ptr(_f64(b)) if b is not None else None,
                    _ptr(x), _ptr(out))
    return out


def conv3d_bwd(grid, batch, W, x, dout, want_din=True):
    nx, ny, nz = grid
    cout, cin = W.shape[0], W.shape[1]
    dW = np.empty(W.shape)
    db = np.empty(cout)
    din = np.empty((batch, cin, nz, ny, nx)) if want_din else None
    lib().or_conv3d_bwd(nx, ny, nz, batch, cin, cout, _ptr(_f64(W)), _ptr(_f64(x)), _ptr(_f64(dout)),
                        _ptr(dW), _ptr(db), _ptr(din) if want_din else None)
    return dW, db, din


def net_input(U):
    """U: [batch, 2, ...] -> per-sample, per-species mean-free potentials (the gauge-free input)."""
    U = _f64(U)
    return U - U.mean(axis=(2, 3, 4), keepdims=True)


def net_forward(grid, params, U, phibar):
    """phi_hat = phibar_I + y_I - <y_I>, y = conv3(tanh(conv2(tanh(conv1(U - <U>)))))."""
    (W1, b1), (W2, b2), (W3, b3) = params
    B = U.shape[0]
    x = net_input(U)
    h1 = np.tanh(conv3d(grid, B, W1, b1, x))
    h2 = np.tanh(conv3d(grid, B, W2, b2, h1))
    y = conv3d(grid, B, W3, b3, h2)
    phi = y - y.mean(axis=(2, 3, 4), keepdims=True) + np.asarray(phibar, dtype=np.float64)[None, :, None, None, None]
    return phi, (x, h1, h2)


def net_loss_grad(grid, params, U, phi_target, phibar):
    """Loss 0.5 * mean((phi_hat - phi*)^2) over all sites, species and samples, and its gradient."""
    (W1, b1), (W2, b2), (W3, b3) = params
    B = U.shape[0]
    phi, (x, h1, h2) = net_forward(grid, params, U, phibar)
    diff = phi - _f64(phi_target)
    n = diff.size
    loss = 0.5 * float((diff * diff).sum()) / n
    g = diff / n
    dy = g - g.mean(axis=(2, 3, 4), keepdims=True)            # through the mean removal
    dW3, db3, dh2 = conv3d_bwd(grid, B, W3, h2, dy)
    dz2 = dh2 * (1.0 - h2 * h2)
    dW2, db2, dh1 = conv3d_bwd(grid, B, W2, h1, dz2)
    dz1 = dh1 * (1.0 - h1 * h1)
    dW1, db1, _ = conv3d_bwd(grid, B, W1, x, dz1, want_din=False)
    return loss, ((dW1, db1), (dW2, db2), (dW3, db3))
