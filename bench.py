#!/usr/bin/env python
"""Benchmark of the coupled LB/DSCF time step on GB300.

Metric: lattice site-updates per second of the whole coupled step (Fletcher-Reeves inversion
with its propagator sweeps, chemical potential, LB collide-stream, convection-diffusion),
V * steps / time, on the 128^3 asymmetric melt (f = 0.3, chi N = 25, N = 64), FP32 form, with
the FP64 form reported beside it.  Inputs are synthetic (seeded noise around the homogeneous
melt) and resident in HBM; the resident state (about 1.1 GB in FP32) is larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed (one process per GPU): every rank advances its own
replica (different seed), weak scaling, no data-path collective; value = all sites updated
by all ranks / the slowest rank's time.  --impl reference times the FP64 CPU oracle (the
baseline arm) on the host cores, rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site-updates/s per LB+DSCF step, 128^3, FP32 vs FP64 same GB300; % HBM roofline"
UNIT = "site-updates/s"
WORKLOAD = "melt128"


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-forms", action="store_true", help="skip the FP64, learned and batched forms")
    ap.add_argument("--forms", default="fp64,fp32_noise,fp32_residual_stop,fp32_self_consistent,fp32_learned,batch48,solution128,net_forward", help="comma-separated forms to report")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_config(cfg):
    return {"workload": f"{cfg['name']}: AB diblock melt, {cfg['grid'][0]}x{cfg['grid'][1]}x{cfg['grid'][2]} periodic, "
                        f"N={cfg['N']}, nA={cfg['nA']}, chi N={cfg['chi'][(0, 1)] * cfg['N']:g}, dt={cfg['dt']} tau, "
                        f"tau_s={cfg['tau_s']}, tau_b={cfg['tau_b']}, LB coupled",
            "grid": list(cfg["grid"]), "N": cfg["N"], "nA": cfg["nA"], "ncg_iters": cfg["ncg_iters"],
            "cn_sweeps": cfg["cn_sweeps"], "hydro": cfg["hydro"],
            "l2": "no flush: the resident step state (G stack + fields, >1 GB) exceeds the 129 MB L2",
            "parallelism": "replicas (one per GPU)"}


# ---------------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------------------------
CPU_SAMPLE_L = 48   # edge of the periodic sub-box both CPU legs time


def oracle_sample_rate(cfg, steps, L=CPU_SAMPLE_L, budget_s=None):
    """Time the FP64 oracle on an L^3 periodic sub-box of the workload (same N, nA, chi, dt,
    relaxation times, inversion and Jacobi counts) for `steps` coupled steps from the seeded
    initial state, stopping early once budget_s seconds have passed (if given).
    Returns (site-updates/s, threads, sample description, steps timed, seconds)."""
    import numpy as np

    import oracle
    from paper_1204_2088_gb300 import inputs
    oracle.build()
    sample = dict(cfg, grid=(L, L, L))
    phi = inputs.initial_fields(sample)
    U = np.zeros_like(phi)
    pop = None
    m0 = phi.reshape(2, -1).sum(1)
    n = 0
    t = time.perf_counter()
    while n < steps:
        st = oracle.step(sample, phi, U, pop, m0)
        phi, U, pop = st["phi"], st["U"], st["pop"]
        n += 1
        if budget_s is not None and time.perf_counter() - t > budget_s:
            break
    dt = time.perf_counter() - t
    desc = (f"{n} coupled steps of the workload on a {L}^3 periodic sub-box (same N, nA, chi, dt, "
            f"tau_s, tau_b, {cfg['ncg_iters']} inversion iterations, {cfg['cn_sweeps']} Jacobi sweeps), "
            f"rate per site")
    return L ** 3 * n / dt, oracle.num_threads(), desc, n, dt


def _cpu_child(cfg, steps, threads, q):
    try:
        if threads:
            os.environ["OMP_NUM_THREADS"] = str(threads)
        q.put(oracle_sample_rate(cfg, steps))
    except Exception as e:  # reported, not raised
        q.put(repr(e))


def _cpu_spawned(cfg, steps, threads=None):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_cpu_child, args=(cfg, steps, threads, q))
    p.start()
    res = q.get(timeout=900)
    p.join(60)
    return None if isinstance(res, str) else res


def cpu_baseline_spawned(cfg, steps=10):
    """The oracle on the host cores, all threads, and on one thread (one step), on the same sub-box
    the reference arm times (processes started with spawn, after the GPU work)."""
    res = _cpu_spawned(cfg, steps)
    if res is None:
        return None
    rate, cores, desc, _, _ = res
    out = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    one = _cpu_spawned(cfg, 1, threads=1)
    if one is not None:
        out["single_thread"] = {"value": one[0], "unit": UNIT, "cores": one[1], "sample": one[2]}
    return out


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1204_2088_gb300 import inputs
    cfg = inputs.workload(WORKLOAD)
    # warm-up steps are not needed by the CPU code; the timed steps run on the same sub-box as the
    # cpu_baseline leg, within about 150 s in all
    rate, cores, desc, n, dt = oracle_sample_rate(cfg, a.steps, budget_s=150.0)
    V = int(cfg["grid"][0] * cfg["grid"][1] * cfg["grid"][2])
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * V / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(cfg),
            "impl": "reference",
            "sample": {"edge": CPU_SAMPLE_L, "steps_timed": n, "ms_per_step": 1e3 * dt / n,
                       "note": "ms_per_step above is the full-size step at the sample's rate per site"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bf16_peak():
    """Dense BF16 burst rate (TFLOP/s) of this GPU model: the measured one, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured burst"
    return 1900.0, "fallback burst"


FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (non-tensor), nominal


def step_bytes_per_site(N, ncg_iters, cn_sweeps, hydro, es=4, evals_per_iter=2):
    """Algorithmic bytes per site of one coupled step (FP32 figures scaled by es / 4): per density
    evaluation the store-forward propagator solve (G_s written and read once, U in, phi out:
    8N + 16) and the inversion's flat passes (about 48); chemical potentials 24; LB collide-stream
    180 with hydrodynamics; convection-diffusion 44 + 40 per Jacobi sweep."""
    b = evals_per_iter * ncg_iters * (8 * N + 16 + 48) + 24 + 44 + 40 * cn_sweeps + (180 if hydro else 0)
    return b * es / 4.0


def step_prop_flops_per_site(N, ncg_iters, evals_per_iter=2):
    """Floating-point operations per site of one step's propagator sweeps (a lower bound of the
    step's arithmetic): per contour step the x, y and z passes of the separable stencil (4 each)
    and the Boltzmann factor (1), and in the backward sweep the quadrature (2): 28 N per density
    evaluation."""
    return evals_per_iter * ncg_iters * 28 * N


def ncu_traffic(kernel_src, N):
    """DRAM bytes per contour step of the propagator sweep from the committed ncu summary, if it
    was taken on the current source of the kernel (hash match); otherwise None."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    ent = d.get("prop_sweep")
    if ent and ent.get("source_sha256_16") == h and ent.get("N") == N:
        return ent.get("dram_bytes_per_contour_step")
    return None


def learned_form(cfg, dev, phi0, timed, world, tuning, steps):
    """FP32 step with the learned predictor.  The network is trained on the GPU (the library's
    kernels, Adam) on (U, phi[U]) pairs generated by the exact method on 32^3 boxes of the same
    physics (three seeds, the first 120 steps of each), then fine-tuned at full size on the
    (U, phi[U]) pairs of 10 exact steps of the full-size run (translation invariant, periodic
    padding).  The full-size run first takes 12 exact steps through the quench transient, then the
    timed steps run with the predictor attached: exact
    corrector every 10 steps, one inversion iteration per predictor step, fallback above the
    tolerance (1e-3; a second run at 2e-3 shows what an accepted predictor gains).  The timed
    region includes the correctors and judgements."""
    import numpy as np
    import torch

    from paper_1204_2088_gb300 import dscf, inputs, replicas

    t_start = time.perf_counter()
    f = cfg["nA"] / cfg["N"]
    phibar = [cfg["phi_p"] * f, cfg["phi_p"] * (1 - f)]
    Us, Ps, held = [], [], None
    for seed in (101, 102, 103, 104):
        small = dict(cfg, grid=(32, 32, 32), seed=seed, name=cfg["name"] + "-train32")
        ctx = dscf.Context(small, dscf.FP32, device=dev)
        ctx.set(dscf.PHI, torch.from_numpy(inputs.initial_fields(small)).float().to(dev))
        u, p = [], []
        for _ in range(120):
            ctx.step(1)
            u.append(ctx.get(dscf.U).clone())
            p.append(ctx.get(dscf.PHIM).clone())
        ctx.close()
        if seed == 104:
            held = (torch.stack(u), torch.stack(p))
        else:
            Us += u
            Ps += p
    U, P = torch.stack(Us), torch.stack(Ps)
    B, iters, lr = 8, 6000, 1e-4
    net = dscf.Net((32, 32, 32), B, seed=3, device=dev)
    one = dscf.Net((32, 32, 32), 1, seed=3, device=dev)
    err = lambda: max((one.forward(held[0][t:t + 1], phibar)[0] - held[1][t]).abs().max().item()
                      for t in range(10, 120, 10))
    e_untrained = err()
    g = torch.Generator().manual_seed(0)
    for it in range(iters):
        idx = torch.randint(0, U.shape[0], (B,), generator=g)
        net.train_step(U[idx], P[idx], phibar, lr=lr * 0.5 * (1 + np.cos(np.pi * it / iters)) + 1e-6)
    one.set_params(net.get_params())
    e_trained = err()
    t_train = time.perf_counter() - t_start
    big = dscf.Net(cfg["grid"], 1, seed=3, device=dev)
    big.set_params(net.get_params())
    del net, one
    # fine-tuning at full size on the exact warm-up steps of the run itself (the pairs the exact
    # method produces anyway): steps 1-10 train, steps 11-12 are held out
    t_ft = time.perf_counter()
    c = dscf.Context(cfg, dscf.FP32, device=dev, tuning=tuning)
    c.set(dscf.PHI, phi0)
    fu, fp = [], []
    for _ in range(12):
        c.step(1)
        fu.append(c.get(dscf.U).clone())
        fp.append(c.get(dscf.PHIM).clone())
    c.close()
    big_err = lambda ts: max((big.forward(fu[t][None], phibar)[0] - fp[t]).abs().max().item() for t in ts)
    e_full0 = big_err((10, 11))
    ft_iters, ft_lr = 300, 2e-5
    gi = torch.Generator().manual_seed(1)
    for it in range(ft_iters):
        t = int(torch.randint(0, 10, (1,), generator=gi))
        big.train_step(fu[t][None], fp[t][None], phibar, lr=ft_lr * 0.5 * (1 + np.cos(np.pi * it / ft_iters)) + 1e-7)
    big.status()
    e_full1 = big_err((10, 11))
    t_ft = time.perf_counter() - t_ft
    del fu, fp
    V = int(np.prod(cfg["grid"]))
    runs = {}
    for tol in (1e-3, 2e-3):
        c = dscf.Context(cfg, dscf.FP32, device=dev, tuning=tuning)
        c.set(dscf.PHI, phi0)
        c.step(12)
        c.set_predictor(big, corrector_every=10, tol=tol, ncg_iters=1)
        c.step(3)
        d0 = c.diagnostics()
        ms = timed(lambda: c.step(steps))
        d = c.diagnostics()
        c.status()
        runs[tol] = {"value": replicas.aggregate_rate([V * steps] * world, [ms]), "ms_per_step": ms / steps,
                     "predictor_steps": d["pred_steps"] - d0["pred_steps"],
                     "exact_steps": d["exact_steps"] - d0["exact_steps"], "last_judged_error": d["pred_err"],
                     "tensor_path": "tcgen05" if big.tensor_path() == 2 else "mma.sync"}
        c.close()
    big.close()
    out = dict(runs[1e-3])
    out.update({"unit": UNIT, "steps": steps, "tol": 1e-3, "corrector_every": 10, "predictor_ncg_iters": 1,
                "exact_warmup_steps": 12, "at_tol_2e-3": runs[2e-3],
                "training": {"pairs": int(U.shape[0]), "grid": [32, 32, 32], "seeds": 3, "iters": iters, "batch": B,
                             "lr": lr, "held_out_max_err_untrained": e_untrained,
                             "held_out_max_err_trained": e_trained, "seconds": t_train},
                "fine_tuning": {"pairs": 10, "grid": list(cfg["grid"]), "iters": ft_iters, "lr": ft_lr,
                                "held_out_max_err_before": e_full0, "held_out_max_err_after": e_full1,
                                "seconds": t_ft}})
    return out


def learned256_form(dev, timed, rank, world, steps=40):
    """The learned predictor on its own workload: the 256^3 symmetric melt (f = 0.5, chi N = 20,
    N = 64), corrector every 10 steps; the exact FP32 step at the same size beside it (these rows
    of 256 sites take the multi-launch contour kernels: a persistent sweep cannot hold 16.8 M sites).
    The network is trained as in the 128^3 form, on 32^3 boxes of this physics, and fine-tuned on
    ten exact steps of the run."""
    import numpy as np
    import torch

    from paper_1204_2088_gb300 import dscf, inputs, replicas

    cfg = inputs.workload("melt256", seed=replicas.rank_seed(5, rank))
    V = int(np.prod(cfg["grid"]))
    phi0 = torch.from_numpy(inputs.initial_fields(cfg)).float().to(dev)
    c = dscf.Context(cfg, dscf.FP32, device=dev)
    d = c.diagnostics()
    tuning = (d["zc"], d["kfuse"])
    c.set(dscf.PHI, phi0)
    c.step(12)
    k = 10
    # the exact steps inside a profiler range (a no-op unless a profiler runs with profiling from
    # start off); the range's ends stay outside the events
    torch.cuda.profiler.start()
    ms = timed(lambda: c.step(k))
    torch.cuda.profiler.stop()
    c.status()
    c.close()
    out = learned_form(cfg, dev, phi0, timed, world, tuning, steps)
    out["exact"] = {"value": replicas.aggregate_rate([V * k] * world, [ms]), "ms_per_step": ms / k, "steps": k,
                    "tuning": list(tuning)}
    out["workload"] = "melt256: AB diblock melt, 256^3, N=64, f=0.5, chi N=20, dt=0.1 tau"
    return out


def residual_stop_form(cfg, dev, phi0, timed, world, tuning, steps):
    """The FP32 step with the inversion stopped on its residual (at most ncg_iters iterations,
    fewer once max|phi* - phi[U]| < tol), measured early after the quench (from step 30) and later
    (from step 300); the steps in between run the fixed count."""
    from paper_1204_2088_gb300 import dscf, replicas
    V = int(cfg["grid"][0] * cfg["grid"][1] * cfg["grid"][2])
    ctx = dscf.Context(cfg, dscf.FP32, device=dev)
    ctx.set(dscf.PHI, phi0)
    out = {"unit": UNIT, "steps": steps}
    done = 0
    for start in (30, 300):
        ctx.set_inversion_tol(0.0)
        ctx.step(start - done)
        done = start
        res = {}
        for tol in (1e-4, 3e-5):
            ctx.set_inversion_tol(tol)
            ctx.step(3)
            ms = timed(lambda: ctx.step(steps))
            its, gend = [], []
            for _ in range(steps):   # iterations actually run, one step at a time (untimed)
                ctx.step(1)
                d = ctx.diagnostics()
                its.append(d["ncg_iters"])
                gend.append(d["gmax_end"])
            ctx.status()
            done += 3 + 2 * steps
            res[f"tol_{tol:g}"] = {"value": replicas.aggregate_rate([V * steps] * world, [ms]), "ms_per_step": ms / steps,
                                   "mean_ncg_iters": sum(its) / len(its), "max_gmax_end": max(gend)}
        out[f"from_step_{start}"] = res
    ctx.close()
    return out


def self_consistent_form(cfg, dev, phi0, timed, world, tuning, steps, tol=1e-5, cap=32):
    """Both starting points of the inversion: the previous potentials and their extrapolation."""
    out = _self_consistent(cfg, dev, phi0, timed, world, tuning, steps, tol, cap, warm=0)
    out["extrapolated_start"] = _self_consistent(cfg, dev, phi0, timed, world, tuning, steps, tol, cap, warm=1)
    return out


def _self_consistent(cfg, dev, phi0, timed, world, tuning, steps, tol, cap, warm):
    """The FP32 step with the inversion run to self-consistency: residual stop at the FP32
    tolerance max|phi* - phi[U]| < 1e-5 with a cap of 32 iterations, measured from step 30 and from
    step 300 after the quench (the first steps, from the cold start U = 0, need the cap).  Reported:
    the rate, the iterations actually run (mean and largest), the largest residual at the end of a
    step, and the whole step against the HBM roofline with the bytes of the iterations run.  With
    warm = 1 every inversion starts from the potentials extrapolated in time (dscf_set_warm_start),
    one extra density evaluation per step."""
    from paper_1204_2088_gb300 import dscf, replicas
    V = int(cfg["grid"][0] * cfg["grid"][1] * cfg["grid"][2])
    ctx = dscf.Context(dict(cfg, ncg_iters=cap), dscf.FP32, device=dev, tuning=tuning)
    ctx.set(dscf.PHI, phi0)
    ctx.set_inversion_tol(tol)
    ctx.set_warm_start(warm)
    out = {"unit": UNIT, "steps": steps, "tol": tol, "ncg_cap": cap, "tuning": list(tuning),
           "start": "extrapolated" if warm else "previous potentials"}
    done = 0
    hbm = peaks()[0]
    for start in (30, 300):
        ctx.step(start - done)
        ms = timed(lambda: ctx.step(steps))
        its, gend = [], []
        for _ in range(steps):   # iterations actually run, one step at a time (untimed)
            ctx.step(1)
            d = ctx.diagnostics()
            its.append(d["ncg_iters"])
            gend.append(d["gmax_end"])
        ctx.status()
        done = start + 2 * steps
        mean_it = sum(its) / len(its)
        b = step_bytes_per_site(cfg["N"], mean_it, cfg["cn_sweeps"], cfg["hydro"])
        if warm:
            b += step_bytes_per_site(cfg["N"], 1, 0, 0, evals_per_iter=1) - step_bytes_per_site(cfg["N"], 0, 0, 0)
        gbps = b * V / (ms / steps * 1e-3) / 1e9
        out[f"from_step_{start}"] = {"value": replicas.aggregate_rate([V * steps] * world, [ms]),
                                     "ms_per_step": ms / steps, "mean_ncg_iters": mean_it,
                                     "max_ncg_iters": max(its), "max_gmax_end": max(gend),
                                     "hbm": {"alg_bytes_per_site": b, "GBps": gbps, "frac": gbps / hbm}}
    ctx.close()
    return out


def solution_form(dev, timed, rank, world, steps):
    """The amphiphilic diblock in solvent at 128^3 (phi_p = 0.12, f_A = 0.3, N = 48, chi_AB N = 30,
    chi_BS N = 35, tau_s = 0.8, tau_b = 1.2, three species), FP32, with the tuning the autotuner
    picks for it."""
    import numpy as np
    import torch

    from paper_1204_2088_gb300 import dscf, inputs, replicas
    cfg = inputs.workload("solution128", seed=replicas.rank_seed(4, rank))
    V = int(np.prod(cfg["grid"]))
    ctx = dscf.Context(cfg, dscf.FP32, device=dev)
    ctx.set(dscf.PHI, torch.from_numpy(inputs.initial_fields(cfg)).float().to(dev))
    ctx.step(3)
    ms = timed(lambda: ctx.step(steps))
    ctx.status()
    d = ctx.diagnostics()
    ctx.close()
    return {"value": replicas.aggregate_rate([V * steps] * world, [ms]), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "workload": "solution128: 128^3, N=48, nA=14, phi_p=0.12, three species",
            "zc": d["zc"], "kfuse": d["kfuse"], "ncg_iters": cfg["ncg_iters"]}


def noise_form(cfg, dev, phi0, timed, world, tuning, steps):
    """The FP32 step with thermal noise (Omega = 400 as in the paper's runs): the composition flux
    noise of Eq. 5 and the fluctuating LB collision of Eq. 13."""
    from paper_1204_2088_gb300 import dscf, replicas
    V = int(cfg["grid"][0] * cfg["grid"][1] * cfg["grid"][2])
    ctx = dscf.Context(cfg, dscf.FP32, device=dev, tuning=tuning)
    ctx.set_noise(400.0, lb_noise=True, seed=2012)
    ctx.set(dscf.PHI, phi0)
    ctx.step(3)
    ms = timed(lambda: ctx.step(steps))
    ctx.status()
    d = ctx.diagnostics()
    ctx.close()
    return {"value": replicas.aggregate_rate([V * steps] * world, [ms]), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "omega": 400.0, "lb_noise": True, "lb_momentum": d["lb_momentum"]}


def net_forward_form(dev, timed, reps=10):
    """The predictor network's forward pass alone at 128^3 (batch 1), on the tcgen05 path and on
    the mma.sync path: mean time of one forward (CUDA events, after a warm-up pass) and the rate in
    TFLOP/s counted on the useful channels (2 x 125 x (2 x 32 + 32 x 32 + 32 x 2) FLOP per site)
    and on the padded ones the kernels compute (2 x 125 x (16 x 32 + 32 x 32 + 32 x 16))."""
    import torch

    from paper_1204_2088_gb300 import dscf
    nx = ny = nz = 128
    net = dscf.Net((nx, ny, nz), 1, seed=1, device=dev)
    g = torch.Generator(device=dev).manual_seed(1)
    U = (torch.randn(1, 2, nz, ny, nx, device=dev, generator=g) * 0.1).float()
    phibar = [0.5, 0.5]
    V = nx * ny * nz
    useful = 2.0 * V * 125 * (2 * 32 + 32 * 32 + 32 * 2)
    padded = 2.0 * V * 125 * (16 * 32 + 32 * 32 + 32 * 16)
    out = {"grid": [nx, ny, nz], "reps": reps}
    for path in (0, 1):
        net.set_tensor_path(path)
        net.forward(U, phibar)
        ms = timed(lambda: [net.forward(U, phibar) for _ in range(reps)]) / reps
        name = "tcgen05" if net.tensor_path() == 2 else "mma.sync"
        out[name] = {"ms": ms, "tflops_useful": useful / ms / 1e9, "tflops_padded": padded / ms / 1e9}
    peak, kind = bf16_peak()
    out["bf16_peak"] = {"tflops": peak, "kind": kind}
    for name in ("tcgen05", "mma.sync"):
        if name in out:
            out[name]["frac_useful"] = out[name]["tflops_useful"] / peak
            out[name]["frac_padded"] = out[name]["tflops_padded"] / peak
    # one more forward on the default path inside a profiler range (a no-op unless a profiler runs
    # with profiling from start off), so that a capture can select exactly its launches
    net.set_tensor_path(0)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.start()
    net.forward(U, phibar)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.stop()
    net.status()
    net.close()
    return out


def batch48_form(dev, timed, rank, world, steps):
    """The 48 mixed-size melts (24 x 48^3, 16 x 64^3, 8 x 96^3) in one FP32 context per rank
    (the replicas split across ranks by site count), one captured graph per step."""
    import numpy as np
    import torch

    from paper_1204_2088_gb300 import dscf, inputs, replicas

    cfgs = inputs.batch48()
    sites = [int(np.prod(c["grid"])) for c in cfgs]
    mine = replicas.partition(sites, world)[rank]
    if not mine:
        ms = timed(lambda: None)
        return None
    sub = [cfgs[i] for i in mine]
    c = dscf.Context(sub, dscf.FP32, device=dev)
    c.set(dscf.PHI, torch.cat([torch.from_numpy(inputs.initial_fields(x)).float().reshape(-1) for x in sub]).to(dev))
    c.step(2)
    # the timed steps inside a profiler range (a no-op unless a profiler runs with profiling from
    # start off); the range's ends stay outside the events
    torch.cuda.profiler.start()
    ms = timed(lambda: c.step(steps))
    torch.cuda.profiler.stop()
    c.status()
    diag = c.diagnostics(0)
    c.close()
    return {"value": replicas.aggregate_rate([sum(sites) * steps], [ms]), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "replicas": len(cfgs), "sites": sum(sites), "zc": diag["zc"], "kfuse": diag["kfuse"]}


def run_ours(a):
    import numpy as np
    import torch

    from paper_1204_2088_gb300 import dscf, inputs, replicas

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = inputs.workload(WORKLOAD, seed=replicas.rank_seed(11, rank))
    V = int(np.prod(cfg["grid"]))
    N = cfg["N"]

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    phi0 = torch.from_numpy(inputs.initial_fields(cfg)).float().to(dev)
    ctx = dscf.Context(cfg, dscf.FP32, device=dev)
    d_init = ctx.diagnostics()
    tuning = (d_init["zc"], d_init["kfuse"])   # the FP32 forms of this workload reuse it
    ctx.set(dscf.PHI, phi0)
    ctx.probe(True)
    ctx.step(a.warmup)
    ctx.status()
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(local)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the profiler range (a no-op unless a profiler runs with profiling from start off) holds
    # exactly the timed steps
    torch.cuda.profiler.start()
    e0.record(stream)
    ctx.step(a.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.stop()
    barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ctx.status()
    ms_max = max_over_ranks(ms)
    sweeps_ms, lb_ms, step_ms = ctx.probe_ms()
    diag = ctx.diagnostics()
    launches = ctx.launches_per_step()
    value = replicas.aggregate_rate([V * a.steps] * world, [ms_max])

    # end to end through the C ABI with host buffers: upload phi, one step, read phi back
    host = torch.empty(tuple(phi0.shape), dtype=torch.float32).pin_memory()
    ctx.get_host(dscf.PHI, host)
    ke2e = max(3, min(a.steps, 30))
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke2e):
        ctx.set(dscf.PHI, host)
        ctx.step(1)
        ctx.get_host(dscf.PHI, host)
    torch.cuda.synchronize(dev)
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    nbytes = host.numel() * host.element_size()
    e2e = {"value": world * V * ke2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": ke2e}
    ctx.close()
    del ctx

    forms = {}
    want = set() if a.no_forms else set(f for f in a.forms.split(",") if f)

    def timed(fn):
        torch.cuda.synchronize(dev)
        barrier()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(e0.elapsed_time(e1))

    alu = None
    if "fp64" in want:
        # measured CUDA-core FMA peaks (the library's dscf_fma_peak), clocks sampled meanwhile
        csamp = ClockSampler(local)
        csamp.start()
        alu = {"fp32_tflops": dscf.fma_peak(dscf.FP32), "fp64_tflops": dscf.fma_peak(dscf.FP64)}
        alu["clocks"] = csamp.stop()
        k64 = max(2, min(10, a.steps // 10))
        c64 = dscf.Context(cfg, dscf.FP64, device=dev)
        c64.set(dscf.PHI, phi0.double())
        c64.probe(True)
        c64.step(2)
        m64 = timed(lambda: c64.step(k64))
        sw64, lb64, st64 = c64.probe_ms()
        b64 = step_bytes_per_site(N, cfg["ncg_iters"], cfg["cn_sweeps"], cfg["hydro"], es=8)
        f64 = step_prop_flops_per_site(N, cfg["ncg_iters"])
        s64 = m64 / k64 * 1e-3
        forms["fp64"] = {"value": replicas.aggregate_rate([V * k64] * world, [m64]), "unit": UNIT,
                         "ms_per_step": m64 / k64, "steps": k64, "prop_sweep_ms_per_launch": sw64 / (2 * N),
                         "lb_ms": lb64,
                         "hbm": {"alg_bytes_per_site": b64, "GBps": b64 * V / s64 / 1e9,
                                 "frac": b64 * V / s64 / 1e9 / peaks()[0]},
                         "fp64_alu": {"prop_flops_per_site": f64, "TFLOPs": f64 * V / s64 / 1e12,
                                      "frac_of_measured": f64 * V / s64 / 1e12 / alu["fp64_tflops"],
                                      "measured_peak_TFLOPs": alu["fp64_tflops"],
                                      "frac_of_nominal": f64 * V / s64 / 1e12 / FP64_NOMINAL_TFLOPS,
                                      "nominal_TFLOPs": FP64_NOMINAL_TFLOPS}}
        c64.close()
        del c64
    if "fp32_noise" in want:
        forms["fp32_noise"] = noise_form(cfg, dev, phi0, timed, world, tuning, max(10, min(a.steps, 20)))
    if "fp32_residual_stop" in want:
        forms["fp32_residual_stop"] = residual_stop_form(cfg, dev, phi0, timed, world, tuning, max(10, min(a.steps, 20)))
    if "fp32_self_consistent" in want:
        forms["fp32_self_consistent"] = self_consistent_form(cfg, dev, phi0, timed, world, tuning, max(10, min(a.steps, 20)))
    if "solution128" in want:
        forms["solution128"] = solution_form(dev, timed, rank, world, max(10, min(a.steps, 20)))
    if "fp32_learned" in want:
        forms["fp32_learned"] = learned_form(cfg, dev, phi0, timed, world, tuning, max(20, min(a.steps, 40)))
    if "fp32_learned_256" in want:   # not in the default list: about four minutes
        forms["fp32_learned_256"] = learned256_form(dev, timed, rank, world)
    if "batch48" in want:
        forms["batch48"] = batch48_form(dev, timed, rank, world, max(3, min(a.steps // 10, 10)))
    if "net_forward" in want:
        forms["net_forward"] = net_forward_form(dev, timed)

    hbm, peak_kind = peaks()
    # Dominant kernel: the propagator sweeps.  The unit is one contour step (the autotuner runs
    # N of them per launch in the persistent kernel, K per launch in the fused one, one in the
    # single-step kernels).  Algorithmic bytes per contour step: the store-forward propagator
    # solve must write G_s once and read it once per density evaluation plus read U and write
    # phi: (8N + 16) B per site per evaluation over its 2N contour steps, i.e. (4 + 8/N) B per
    # site per step (FP32).
    per_launch_s = sweeps_ms * 1e-3 / (2 * N)
    alg_bytes = (4.0 + 8.0 / N) * V
    achieved = alg_bytes / per_launch_s / 1e9
    traffic = ncu_traffic(os.path.join(ROOT, "paper_1204_2088_gb300", "csrc", "dscf_pers.cu"), N)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic,
            "kernel": {0: "k_prop_pers (persistent sweep)", 1: "k_prop (single step)"}.get(
                diag["kfuse"], f"k_prop_fused (K={diag['kfuse']})") + "; unit = one contour step",
            "alg_bytes_per_launch": alg_bytes, "ms_per_launch": per_launch_s * 1e3, "peak_kind": peak_kind}
    lb_alg = 180.0 * V
    bstep = step_bytes_per_site(N, cfg["ncg_iters"], cfg["cn_sweeps"], cfg["hydro"])
    sstep = ms_max / a.steps * 1e-3
    kernels = {"step": {"alg_bytes_per_site": bstep, "GBps": bstep * V / sstep / 1e9,
                        "hbm_frac": bstep * V / sstep / 1e9 / hbm},
               "prop_sweep": {"ms_per_launch": per_launch_s * 1e3, "GBps": achieved},
               "lb_collide_stream": {"ms": lb_ms, "alg_bytes": lb_alg,
                                     "GBps": lb_alg / (lb_ms * 1e-3) / 1e9 if lb_ms > 0 else None},
               "step_ms_probe": step_ms}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline_spawned(cfg)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(cfg), "e2e": e2e, "gpu_launches": int(launches * a.steps),
                "roofline": roof, "cpu_baseline": cpu, "clocks": clk, "forms": forms, "kernels": kernels,
                "alu_peaks": alu,
                "ncg": {"iters": diag["ncg_iters"], "line_search_evals_per_iter": 1,
                        "gmax_start": diag["gmax_start"], "gmax_end": diag["gmax_end"]},
                "umax": diag["umax"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = args_()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
