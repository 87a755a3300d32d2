"""Quench runs of the paper's ordering workloads (Sec. 3): a homogeneous melt or solution is
quenched into the ordered region and the free energy F, the order parameter S and the
segregation are recorded along the run, with hydrodynamics (LB coupled) and without (the
diffusion-only model, u = 0), with the same seeds and noise.

    python -m paper_1204_2088_gb300.quench --system A8B8 --grid 48 --steps 30000 --every 1000 \
        --seeds 1 2 --out quench.jsonl

Systems (synthetic stand-ins for the paper's runs, Sec. 3):
  A8B8    symmetric melt, N = 16, f = 0.5, chi^0_AB = 1.0 (chi N = 16): lamellae
  A5B11   asymmetric melt, N = 16, f = 5/16, chi^0_AB = 1.3 (chi N = 20.8): cylinders (Fig. 2b)
  A2B8S   A2B8 in solvent, copolymer fraction 0.2, chi^0_AB = 2.3, chi^0_BS = 2.4, chi^0_AS = 0.25
Protocol: 48^3 (the paper's Fig. 2 box), tau_s = tau_b = 1, six inversion iterations per step,
dt = 0.1 tau, no thermal noise by default (--omega sets the noise parameter, --lb-noise adds the LB
modes).  With this scheme's explicit force coupling these short chains (N = 16, chi N = 16) are
unstable with hydrodynamics at dt = 0.2 tau even without noise; with noise (Omega = 100 or 400)
the explicit noise step drives the minority composition of a strongly segregated 48^3 box through
zero within a few thousand steps, where the inversion cannot follow.  A run that breaks down ends
with an "error" record.
With --batch every seed and every (tau_s, tau_b) pair of --viscosities runs as one replica of a
single context (all replicas in the same launches and one CUDA graph per step), so a protocol of
several seeds and viscosities costs about one larger run; each replica's record carries its seed
and relaxation times.
Every record is one JSON line: system, hydro, seed, step, time (tau), F, S, segregation, the
Minkowski functionals of the B beads at threshold 0.2 (V, S, 2B, chi), for the solution the
fraction of the solvent enclosed by {phi_B > 0.2} and the number of solvent components, and the
mean milliseconds per step of the segment before it.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np
import torch

from . import dscf, inputs


def system_cfg(name: str, grid: int, seed: int, hydro: int) -> dict:
    g = (grid, grid, grid)
    if name == "A8B8":
        cfg = inputs.melt(g, 16, 0.5, 16.0, 1.0, 1.0, 0.01, seed, dt=0.1, hydro=hydro, ncg_iters=6, name=name)
    elif name == "A5B11":
        cfg = inputs.melt(g, 16, 5 / 16, 20.8, 1.0, 1.0, 0.01, seed, dt=0.1, hydro=hydro, ncg_iters=6, name=name)
    elif name == "A2B8S":
        cfg = inputs.solution(g, 10, 0.2, 0.2, 23.0, 24.0, 2.5, 1.0, 1.0, 0.01, seed, dt=0.1, hydro=hydro,
                              ncg_iters=6, name=name)
    else:
        raise KeyError(name)
    return cfg


def run(name: str, grid: int, steps: int, every: int, seed: int, hydro: int, omega: float = 0.0,
        lb_noise: bool = False, precision=dscf.FP32, viscosity=None):
    """Yields one record per `every` steps (and the initial state); a record with "error" ends a
    run that broke down (a non-finite value, reported by the library's status check).
    viscosity: (tau_s, tau_b) in place of the system's relaxation times."""
    cfg = system_cfg(name, grid, seed, hydro)
    if viscosity is not None:
        cfg = dict(cfg, tau_s=float(viscosity[0]), tau_b=float(viscosity[1]))
    ctx = dscf.Context(cfg, precision)
    ctx.set_noise(omega, lb_noise=bool(hydro and lb_noise), seed=1000 + seed)
    dt = torch.float32 if precision == dscf.FP32 else torch.float64
    ctx.set(dscf.PHI, torch.from_numpy(inputs.initial_fields(cfg)).to(dt).cuda())
    done = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    base = {"system": name, "grid": grid, "hydro": hydro, "seed": seed, "omega": omega}
    ms = None
    try:
        while True:
            ob = ctx.observables()
            mk = ctx.minkowski(1, 0.2)   # the B beads at the paper's threshold
            rec = dict(base, step=done, time=done * cfg["dt"], F=ob["free_energy"], S=ob["order_parameter"],
                       segregation=ob["segregation"], minkowski_B=mk)
            if cfg["ns"] == 3:
                rec["trapped_solvent"], rec["solvent_components"] = ctx.trapped_solvent(0.2)
            if ms is not None:
                rec["ms_per_step"] = ms
            yield rec
            if done >= steps:
                break
            k = min(every, steps - done)
            e0.record()
            ctx.step(k)
            e1.record()
            torch.cuda.synchronize()
            ctx.status()
            ms = e0.elapsed_time(e1) / k
            done += k
    except dscf.DSCFError as e:
        yield dict(base, step=done, error=str(e))
    finally:
        ctx.close()


def run_batch(name: str, grid: int, steps: int, every: int, seeds, hydro: int, viscosities=((1.0, 1.0),),
              omega: float = 0.0, lb_noise: bool = False, precision=dscf.FP32):
    """As run(), for every (seed, (tau_s, tau_b)) pair at once as the replicas of one context.
    Yields one record per replica per `every` steps; an "error" record (one per replica) ends the
    batch.  Without noise each replica follows its solo run; with noise every replica draws its
    own stream (keyed by its place in the batch), so noisy batch runs are other samples than the
    solo runs of the same seeds."""
    cfgs, tags = [], []
    for ts, tb in viscosities:
        for seed in seeds:
            cfg = dict(system_cfg(name, grid, seed, hydro), tau_s=float(ts), tau_b=float(tb))
            cfgs.append(cfg)
            tags.append({"system": name, "grid": grid, "hydro": hydro, "seed": seed, "omega": omega,
                         "tau_s": float(ts), "tau_b": float(tb)})
    ctx = dscf.Context(cfgs, precision)
    ctx.set_noise(omega, lb_noise=bool(hydro and lb_noise), seed=1000 + int(seeds[0]))
    dt = torch.float32 if precision == dscf.FP32 else torch.float64
    ctx.set(dscf.PHI, torch.cat([torch.from_numpy(inputs.initial_fields(c)).to(dt).reshape(-1) for c in cfgs]).cuda())
    done, ms = 0, None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        while True:
            for r, (cfg, tag) in enumerate(zip(cfgs, tags)):
                ob = ctx.observables(r)
                rec = dict(tag, step=done, time=done * cfg["dt"], F=ob["free_energy"], S=ob["order_parameter"],
                           segregation=ob["segregation"], minkowski_B=ctx.minkowski(1, 0.2, replica=r))
                if cfg["ns"] == 3:
                    rec["trapped_solvent"], rec["solvent_components"] = ctx.trapped_solvent(0.2, replica=r)
                if ms is not None:
                    rec["ms_per_step"] = ms
                yield rec
            if done >= steps:
                break
            k = min(every, steps - done)
            e0.record()
            ctx.step(k)
            e1.record()
            torch.cuda.synchronize()
            ctx.status()
            ms = e0.elapsed_time(e1) / k
            done += k
    except dscf.DSCFError as e:
        for tag in tags:
            yield dict(tag, step=done, error=str(e))
    finally:
        ctx.close()


def summarize(records):
    """Mean and sample standard deviation over seeds of F, S and segregation, per condition
    (system, grid, hydro, tau_s, tau_b, omega) and time; runs that ended in an "error" record are
    left out from that record on.  Returns a list of dicts sorted by condition and time."""
    groups = {}
    for r in records:
        if "error" in r:
            continue
        key = (r["system"], r["grid"], r["hydro"], r.get("tau_s"), r.get("tau_b"), r.get("omega", 0.0), r["time"])
        groups.setdefault(key, []).append(r)
    out = []
    for key in sorted(groups, key=lambda k: tuple((x is None, x) for x in k)):
        rs = groups[key]
        row = dict(zip(("system", "grid", "hydro", "tau_s", "tau_b", "omega", "time"), key), seeds=len(rs))
        for q in ("F", "S", "segregation"):
            v = np.array([r[q] for r in rs], dtype=np.float64)
            row[q] = float(v.mean())
            row[q + "_std"] = float(v.std(ddof=1)) if len(v) > 1 else 0.0
        out.append(row)
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--system", default="A8B8", choices=["A8B8", "A5B11", "A2B8S"])
    ap.add_argument("--grid", type=int, default=48)
    ap.add_argument("--steps", type=int, default=30000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--seeds", type=int, nargs="+", default=[1])
    ap.add_argument("--omega", type=float, default=0.0, help="noise parameter (0: no thermal noise)")
    ap.add_argument("--lb-noise", action="store_true")
    ap.add_argument("--batch", action="store_true", help="all seeds and viscosities as replicas of one context")
    ap.add_argument("--viscosities", type=float, nargs="+", default=[1.0, 1.0],
                    help="tau_s tau_b pairs for the hydrodynamic runs of --batch")
    ap.add_argument("--out", default="-")
    ap.add_argument("--summarize", metavar="JSONL", help="print mean and spread over seeds of a finished run file")
    a = ap.parse_args(argv)
    if a.summarize:
        with open(a.summarize) as f:
            recs = [json.loads(line) for line in f if line.strip()]
        for row in summarize(recs):
            print(json.dumps(row))
        return 0
    if len(a.viscosities) % 2:
        ap.error("--viscosities takes tau_s tau_b pairs")
    visc = list(zip(a.viscosities[0::2], a.viscosities[1::2]))
    out = sys.stdout if a.out == "-" else open(a.out, "w")
    if a.batch:
        runs = [run_batch(a.system, a.grid, a.steps, a.every, a.seeds, 0, visc[:1], a.omega, a.lb_noise),
                run_batch(a.system, a.grid, a.steps, a.every, a.seeds, 1, visc, a.omega, a.lb_noise)]
    else:
        runs = [run(a.system, a.grid, a.steps, a.every, seed, hydro, a.omega, a.lb_noise)
                for seed in a.seeds for hydro in (0, 1)]
    for it in runs:
        for r in it:
            out.write(json.dumps(r) + "\n")
            out.flush()
    if out is not sys.stdout:
        out.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
