"""Python binding of libdscf.so (include/dscf.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only builds the parameter
structs, allocates the device workspace with PyTorch (the only allocator), passes raw
pointers and the current CUDA stream, and wraps results as tensors.  There is no CPU
fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdscf.so")

DSCF_OK = 0
ERRORS = {-1: "DSCF_ERR_ARG", -2: "DSCF_ERR_CUDA", -3: "DSCF_ERR_OOM", -4: "DSCF_ERR_TIMEOUT",
          -5: "DSCF_ERR_NUMERIC", -6: "DSCF_ERR_STATE", -7: "DSCF_ERR_NOCONVERGE"}
FP64, FP32 = 0, 1
PHI, U, MU, VEL, POP, PHIM = 0, 1, 2, 3, 4, 5


class DSCFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """Mirror of dscf_params."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("ns", ctypes.c_int32), ("N", ctypes.c_int32), ("nA", ctypes.c_int32),
        ("phi_p", ctypes.c_double), ("chi", ctypes.c_double * 9), ("kappa", ctypes.c_double),
        ("a", ctypes.c_double), ("dt", ctypes.c_double), ("M", ctypes.c_double),
        ("tau_s", ctypes.c_double), ("tau_b", ctypes.c_double), ("rho0", ctypes.c_double),
        ("hydro", ctypes.c_int32), ("ncg_iters", ctypes.c_int32), ("cn_sweeps", ctypes.c_int32),
        ("phi_floor", ctypes.c_double),
    ]


_lib = None


def load():
    """Load libdscf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
    P = ctypes.POINTER(Params)
    sigs = {
        "dscf_workspace_bytes": (sz, [P, i32, i32]),
        "dscf_init": (ctypes.c_int, [P, i32, i32, vp, sz, vp, ctypes.POINTER(vp)]),
        "dscf_init_tuned": (ctypes.c_int, [P, i32, i32, vp, sz, vp, i32, i32, ctypes.POINTER(vp)]),
        "dscf_step": (ctypes.c_int, [vp, i32]),
        "dscf_densities": (ctypes.c_int, [vp, vp, vp]),
        "lb_step": (ctypes.c_int, [vp, vp, i32]),
        "dscf_get_fields": (ctypes.c_int, [vp, i32, vp, i32]),
        "dscf_set_fields": (ctypes.c_int, [vp, i32, vp, i32]),
        "dscf_diagnostics": (ctypes.c_int, [vp, i32, ctypes.POINTER(ctypes.c_double)]),
        "dscf_status": (ctypes.c_int, [vp]),
        "dscf_free": (ctypes.c_int, [vp]),
        "dscf_last_error": (ctypes.c_char_p, [vp]),
        "dscf_launches_per_step": (ctypes.c_int64, [vp]),
        "dscf_probe": (ctypes.c_int, [vp, i32]),
        "dscf_probe_ms": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float)]),
        "dscf_densities_static": (ctypes.c_int, [P, i32, vp, vp, vp]),
        "dscf_set_tuning": (ctypes.c_int, [vp, i32, i32]),
        "dscf_net_workspace_bytes": (sz, [i32, i32, i32, i32]),
        "dscf_net_init": (ctypes.c_int, [i32, i32, i32, i32, ctypes.c_uint64, vp, sz, vp, ctypes.POINTER(vp)]),
        "dscf_net_forward": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_double), vp]),
        "dscf_net_gradient": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp,
                                             ctypes.POINTER(ctypes.c_double), vp]),
        "dscf_net_train_step": (ctypes.c_int, [vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp, ctypes.c_float,
                                               ctypes.POINTER(ctypes.c_double)]),
        "dscf_net_get_params": (ctypes.c_int, [vp, vp]),
        "dscf_net_set_params": (ctypes.c_int, [vp, vp]),
        "dscf_net_num_params": (ctypes.c_int64, []),
        "dscf_net_free": (ctypes.c_int, [vp]),
        "dscf_net_last_error": (ctypes.c_char_p, [vp]),
        "dscf_set_predictor": (ctypes.c_int, [vp, vp, i32, ctypes.c_double, i32]),
        "dscf_set_wait_limit": (ctypes.c_int, [vp, i32]),
        "dscf_set_inversion_tol": (ctypes.c_int, [vp, ctypes.c_double]),
        "dscf_set_warm_start": (ctypes.c_int, [vp, i32]),
        "dscf_set_noise": (ctypes.c_int, [vp, ctypes.c_double, i32, ctypes.c_uint64]),
        "dscf_minkowski": (ctypes.c_int, [vp, i32, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]),
        "dscf_trapped_solvent": (ctypes.c_int, [vp, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "dscf_observables": (ctypes.c_int, [vp, i32, ctypes.POINTER(ctypes.c_double)]),
        "dscf_net_set_tensor_path": (ctypes.c_int, [vp, i32]),
        "dscf_net_tensor_path": (i32, [vp]),
        "dscf_net_status": (ctypes.c_int, [vp]),
        "dscf_inject_lag": (ctypes.c_int, [vp, i32]),
        "dscf_fma_peak": (ctypes.c_int, [i32, vp, ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def make_params(cfg: dict) -> Params:
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
    p.dt = cfg.get("dt", 0.2)
    p.M = cfg.get("M", 1.0)
    p.tau_s = cfg.get("tau_s", 1.0)
    p.tau_b = cfg.get("tau_b", 1.0)
    p.rho0 = cfg.get("rho0", 1.0)
    p.hydro = cfg.get("hydro", 1)
    p.ncg_iters = cfg.get("ncg_iters", 4)
    p.cn_sweeps = cfg.get("cn_sweeps", 8)
    p.phi_floor = cfg.get("phi_floor", 1e-6)
    return p


def workspace_bytes(cfgs, precision=FP64) -> int:
    cfgs = [cfgs] if isinstance(cfgs, dict) else list(cfgs)
    arr = (Params * len(cfgs))(*[make_params(c) for c in cfgs])
    return int(load().dscf_workspace_bytes(arr, len(cfgs), precision))


STATIC_SCRATCH_BYTES = 64 * 1024 * 1024


def densities_static(cfg: dict, U: torch.Tensor, out: torch.Tensor, precision=FP64, stream=None):
    """phi[U] through dscf_densities_static: for callers that cannot allocate device memory.

    U and out are caller-owned device tensors ([ns, nz, ny, nx], contiguous, in the precision's
    dtype); nothing is allocated here or in the library.  Raises DSCFError on an error code."""
    lib = load()
    want = torch.float64 if precision == FP64 else torch.float32
    for t in (U, out):
        if t.device.type != "cuda" or t.dtype != want or not t.is_contiguous():
            raise ValueError("U and out must be contiguous CUDA tensors of the precision's dtype")
    p = make_params(cfg)
    s = stream if stream is not None else torch.cuda.current_stream(U.device)
    rc = lib.dscf_densities_static(ctypes.byref(p), precision, ctypes.c_void_p(U.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if rc != DSCF_OK:
        raise DSCFError(rc, lib.dscf_last_error(None).decode())
    return out


def fma_peak(precision=FP32, stream=None) -> float:
    """Measured FMA throughput of the current device's CUDA cores in TFLOP/s (dscf_fma_peak)."""
    lib = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double()
    rc = lib.dscf_fma_peak(int(precision), ctypes.c_void_p(s.cuda_stream), ctypes.byref(out))
    if rc != DSCF_OK:
        raise DSCFError(rc, lib.dscf_last_error(None).decode())
    return out.value


def _tuning_key(cfgs, precision, device) -> str:
    name = torch.cuda.get_device_name(device)
    shapes = [[list(c["grid"]), c.get("ns", 2), int(c["N"])] for c in cfgs]
    return json.dumps([name, int(precision), shapes])


def _tuning_cache_read(path) -> dict:
    try:
        with open(path) as f:
            return {k: tuple(v) for k, v in json.load(f).items()}
    except (OSError, ValueError):
        return {}


def _tuning_cache_write(path, key, tuning):
    d = _tuning_cache_read(path)
    d[key] = list(tuning)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump({k: list(v) for k, v in d.items()}, f, indent=1)
    os.replace(tmp, path)


class Context:
    """One library context: n replicas (a dict or a list of dicts), one precision, one device.

    Field tensors use the layout of include/dscf.h: for one replica [ncomp, nz, ny, nx], for
    several the replica blocks concatenated into one flat tensor."""

    def __init__(self, cfgs, precision=FP64, device=None, stream=None, tuning=None, tuning_cache=None):
        """tuning: (zc, kfuse) to use instead of the autotuner; tuning_cache: path of a JSON file
        mapping (device, precision, replica shapes) to the tuning the autotuner chose, read before
        and written after the autotuner runs."""
        self.lib = load()
        self.cfgs = [cfgs] if isinstance(cfgs, dict) else list(cfgs)
        self.n = len(self.cfgs)
        self.precision = precision
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._params = (Params * self.n)(*[make_params(c) for c in self.cfgs])
        nbytes = self.lib.dscf_workspace_bytes(self._params, self.n, precision)
        if nbytes == 0:
            raise DSCFError(-1, "invalid parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        key = None
        if tuning is None and tuning_cache is not None:
            key = _tuning_key(self.cfgs, precision, self.device)
            tuning = _tuning_cache_read(tuning_cache).get(key)
        h = ctypes.c_void_p()
        zc, kfuse = (int(tuning[0]), int(tuning[1])) if tuning is not None else (-1, -1)
        rc = self.lib.dscf_init_tuned(self._params, self.n, precision, ctypes.c_void_p(self.workspace.data_ptr()),
                                      nbytes, ctypes.c_void_p(self.stream.cuda_stream), zc, kfuse, ctypes.byref(h))
        if rc != DSCF_OK:
            raise DSCFError(rc, self.lib.dscf_last_error(None).decode())
        self.h = h
        if key is not None and tuning is None:
            d = self.diagnostics()
            _tuning_cache_write(tuning_cache, key, (d["zc"], d["kfuse"]))
        self.V = [c["grid"][0] * c["grid"][1] * c["grid"][2] for c in self.cfgs]
        self.ns = [c.get("ns", 2) for c in self.cfgs]

    # -- helpers ---------------------------------------------------------------------------
    def _check(self, rc):
        if rc != DSCF_OK:
            raise DSCFError(rc, self.lib.dscf_last_error(self.h).decode())

    def _ncomp(self, which):
        return {VEL: [3] * self.n, POP: [19] * self.n}.get(which, self.ns)

    def _shape(self, which):
        nc = self._ncomp(which)
        if self.n == 1:
            nx, ny, nz = self.cfgs[0]["grid"]
            return (nc[0], nz, ny, nx)
        return (sum(c * v for c, v in zip(nc, self.V)),)

    def _as_field(self, t, which):
        t = torch.as_tensor(t)
        if t.device.type == "cpu":
            t = t.to(self.device)
        t = t.to(self.dtype).contiguous()
        if t.numel() != int(np.prod(self._shape(which))):
            raise ValueError(f"field has {t.numel()} elements, expected {int(np.prod(self._shape(which)))}")
        return t

    # -- API -------------------------------------------------------------------------------
    def step(self, n_steps=1):
        self._check(self.lib.dscf_step(self.h, int(n_steps)))

    def densities(self, U):
        Ud = self._as_field(U, PHI)
        out = torch.empty(self._shape(PHI), dtype=self.dtype, device=self.device)
        self._check(self.lib.dscf_densities(self.h, ctypes.c_void_p(Ud.data_ptr()), ctypes.c_void_p(out.data_ptr())))
        return out

    def lb_step(self, force=None, n_steps=1):
        ptr = None
        if force is not None:
            force = self._as_field(force, VEL)
            ptr = ctypes.c_void_p(force.data_ptr())
        self._check(self.lib.lb_step(self.h, ptr, int(n_steps)))
        self._keep = force

    def get(self, which):
        out = torch.empty(self._shape(which), dtype=self.dtype, device=self.device)
        self._check(self.lib.dscf_get_fields(self.h, which, ctypes.c_void_p(out.data_ptr()), 0))
        return out

    def get_host(self, which, out: torch.Tensor):
        """Copy a field into a (preferably pinned) host tensor; synchronises."""
        assert out.device.type == "cpu" and out.dtype == self.dtype and out.is_contiguous()
        self._check(self.lib.dscf_get_fields(self.h, which, ctypes.c_void_p(out.data_ptr()), 1))
        return out

    def set(self, which, t):
        """Field from a device tensor, or from a host tensor: a pinned host tensor of the context's
        dtype is copied asynchronously on the context's stream (the caller keeps it unchanged until
        the next synchronising call), any other host tensor is staged and waited for."""
        if isinstance(t, torch.Tensor) and t.device.type == "cpu":
            src = t.to(self.dtype).contiguous()
            self._check(self.lib.dscf_set_fields(self.h, which, ctypes.c_void_p(src.data_ptr()), 1))
            if src.data_ptr() == t.data_ptr() and t.is_pinned():
                self._keep = src
            else:
                self.stream.synchronize()
            return
        src = self._as_field(t, which)
        self._check(self.lib.dscf_set_fields(self.h, which, ctypes.c_void_p(src.data_ptr()), 0))
        self._keep = src

    def diagnostics(self, replica=0):
        out = (ctypes.c_double * 24)()
        self._check(self.lib.dscf_diagnostics(self.h, replica, out))
        v = list(out)
        return {"mass": v[0:3], "mass_drift": v[3:6], "lb_mass": v[6], "lb_momentum": v[7:10],
                "umax": v[10], "Q": v[11], "QS": v[12], "ncg_iters": int(v[13]), "gg_start": v[14],
                "gmax_start": v[15], "gg_end": v[16], "gmax_end": v[17], "steps": int(v[18]),
                "zc": int(v[19]), "kfuse": int(v[20]), "pred_steps": int(v[21]), "exact_steps": int(v[22]),
                "pred_err": v[23]}

    def status(self):
        self._check(self.lib.dscf_status(self.h))

    def observables(self, replica=0):
        """Free energy per site, order parameter S and segregation of a replica (synchronises)."""
        out = (ctypes.c_double * 3)()
        self._check(self.lib.dscf_observables(self.h, int(replica), out))
        return {"free_energy": out[0], "order_parameter": out[1], "segregation": out[2]}

    def minkowski_counts(self, species, threshold=0.2, replica=0):
        """(n_c, n_f, n_e, n_v) of the body {phi_species > threshold}."""
        out = (ctypes.c_int64 * 4)()
        self._check(self.lib.dscf_minkowski(self.h, int(replica), int(species), float(threshold), out))
        return tuple(out)

    def minkowski(self, species, threshold=0.2, replica=0):
        """Volume, surface, 2 x integral mean curvature (lattice units) and Euler characteristic."""
        nc, nf, ne, nv = self.minkowski_counts(species, threshold, replica)
        return {"V": nc, "S": -6 * nc + 2 * nf, "B2": 3 * nc - 2 * nf + ne, "chi": -nc + nf - ne + nv}

    def trapped_solvent(self, threshold=0.2, replica=0):
        """(fraction of the solvent enclosed by {phi_B > threshold}, number of components)."""
        out = (ctypes.c_double * 2)()
        self._check(self.lib.dscf_trapped_solvent(self.h, int(replica), float(threshold), out))
        return out[0], int(out[1])

    def set_predictor(self, net, corrector_every=10, tol=1e-3, ncg_iters=0):
        """Attach a trained Net (same grid, batch 1) as the density map of the inversion, judged
        by an exact corrector step every corrector_every steps; None detaches."""
        self._check(self.lib.dscf_set_predictor(self.h, net.h if net is not None else None, int(corrector_every),
                                                float(tol), int(ncg_iters)))
        self._net = net

    def set_wait_limit(self, polls):
        """Polls a persistent sweep spends on a neighbour before it reports DSCF_ERR_TIMEOUT."""
        self._check(self.lib.dscf_set_wait_limit(self.h, int(polls)))

    def inject_lag(self, brick):
        """Test hook: make brick's step counter lag so the next persistent sweep times out."""
        self._check(self.lib.dscf_inject_lag(self.h, int(brick)))

    def set_noise(self, omega, lb_noise=True, seed=0):
        """Thermal noise with noise parameter Omega (0: off); lb_noise also the LB modes."""
        self._check(self.lib.dscf_set_noise(self.h, float(omega), int(bool(lb_noise)), int(seed)))

    def set_inversion_tol(self, tol):
        """Residual stop of the inversion: at most ncg_iters iterations, fewer once max|phi* - phi[U]|
        < tol (0: fixed count)."""
        self._check(self.lib.dscf_set_inversion_tol(self.h, float(tol)))

    def set_warm_start(self, mode):
        """0: the inversion starts from the previous potentials; 1: from their linear
        extrapolation in time (see dscf_set_warm_start)."""
        self._check(self.lib.dscf_set_warm_start(self.h, int(mode)))

    def set_tuning(self, zc, kfuse):
        self._check(self.lib.dscf_set_tuning(self.h, int(zc), int(kfuse)))

    def probe(self, enable=True):
        self._check(self.lib.dscf_probe(self.h, 1 if enable else 0))

    def probe_ms(self):
        """(contour sweeps of one gradient evaluation, LB launch, whole step) of the last step, ms."""
        out = (ctypes.c_float * 3)()
        self._check(self.lib.dscf_probe_ms(self.h, out))
        return tuple(float(v) for v in out)

    def launches_per_step(self):
        return int(self.lib.dscf_launches_per_step(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dscf_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """Learned density-map predictor (see include/dscf.h): batch x [2][nz][ny][nx] FP32 fields."""

    def __init__(self, grid, batch=1, seed=1, device=None, stream=None):
        self.lib = load()
        self.grid = tuple(int(g) for g in grid)
        self.batch = int(batch)
        nx, ny, nz = self.grid
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = self.lib.dscf_net_workspace_bytes(nx, ny, nz, self.batch)
        if nbytes == 0:
            raise DSCFError(-1, "network grid needs nx a multiple of 16")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        rc = self.lib.dscf_net_init(nx, ny, nz, self.batch, seed, ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != DSCF_OK:
            raise DSCFError(rc, self.lib.dscf_net_last_error(None).decode())
        self.h = h
        self.nparam = int(self.lib.dscf_net_num_params())
        self.shape = (self.batch, 2, nz, ny, nx)
        self._work = torch.empty(self.shape, dtype=torch.float32, device=self.device)

    def _check(self, rc):
        if rc != DSCF_OK:
            raise DSCFError(rc, self.lib.dscf_net_last_error(self.h).decode())

    def _f32(self, t):
        t = torch.as_tensor(t).to(self.device, torch.float32).contiguous()
        if t.numel() != int(np.prod(self.shape)):
            raise ValueError("field shape does not match the network context")
        return t

    @staticmethod
    def _pb(phibar):
        return (ctypes.c_double * 2)(float(phibar[0]), float(phibar[1]))

    def forward(self, U, phibar):
        U = self._f32(U)
        out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        self._check(self.lib.dscf_net_forward(self.h, ctypes.c_void_p(U.data_ptr()), self._pb(phibar),
                                              ctypes.c_void_p(out.data_ptr())))
        return out

    def gradient(self, U, target, phibar):
        U, target = self._f32(U), self._f32(target)
        g = torch.empty(self.nparam, dtype=torch.float32, device=self.device)
        loss = ctypes.c_double()
        self._check(self.lib.dscf_net_gradient(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                               self._pb(phibar), ctypes.c_void_p(self._work.data_ptr()),
                                               ctypes.byref(loss), ctypes.c_void_p(g.data_ptr())))
        return loss.value, g

    def train_step(self, U, target, phibar, lr=1e-3, want_loss=False):
        U, target = self._f32(U), self._f32(target)
        loss = ctypes.c_double()
        self._check(self.lib.dscf_net_train_step(self.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(target.data_ptr()),
                                                 self._pb(phibar), ctypes.c_void_p(self._work.data_ptr()), float(lr),
                                                 ctypes.byref(loss) if want_loss else None))
        self._keep = (U, target)
        return loss.value if want_loss else None

    def set_tensor_path(self, path):
        """0: tcgen05 forward where the grid allows it (default), 1: mma.sync only."""
        self._check(self.lib.dscf_net_set_tensor_path(self.h, int(path)))

    def tensor_path(self):
        """2 if the forward convolutions run on tcgen05, 1 for mma.sync."""
        return int(self.lib.dscf_net_tensor_path(self.h))

    def status(self):
        self._check(self.lib.dscf_net_status(self.h))

    def get_params(self):
        p = torch.empty(self.nparam, dtype=torch.float32, device=self.device)
        self._check(self.lib.dscf_net_get_params(self.h, ctypes.c_void_p(p.data_ptr())))
        return p

    def set_params(self, p):
        p = torch.as_tensor(p).to(self.device, torch.float32).contiguous()
        self._check(self.lib.dscf_net_set_params(self.h, ctypes.c_void_p(p.data_ptr())))
        self._keep = p

    def close(self):
        if getattr(self, "h", None):
            self.lib.dscf_net_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def net_params_split(p):
    """FP32 parameter vector -> [(W1, b1), (W2, b2), (W3, b3)] numpy arrays."""
    p = np.asarray(p, dtype=np.float64)
    out, off = [], 0
    for cin, cout in ((2, 32), (32, 32), (32, 2)):
        n = cout * cin * 125
        out.append([p[off:off + n].reshape(cout, cin, 125), p[off + n:off + n + cout]])
        off += n + cout
    return out
