"""Benchmark of the PIC-MCC particle cycle on one GB300 (or N independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbpic|reference]

Workload: the 2D capacitively coupled discharge (512 x 16 square cells, plates at x = 0 with
200 V at 13.56 MHz and x = 6.7 cm grounded, periodic in y, electrons and 4 amu ions, 100
macro-particles per cell and species = 2 x 819,200, Maxwellian 2.5 eV / 0.026 eV, analytic
elastic + ionization cross sections, dt = 1/(400 f)), FP32 particle state.  One step is the
whole cycle: NGP deposit, multigrid Poisson, corner field, fused gather/push/locate/MCC,
cell-list update.  Inputs are resident in HBM; L2 is flushed (256 MiB write) before every
timed step, outside the timed events.

Prints one JSON line: particle-steps/s (whole job), the roofline of the dominant particle
kernel (the move pass of the fused push), the oracle's CPU baseline on a bounded sample,
the end-to-end rate through the C ABI with host buffers, clocks and kernel launches.
`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ccp-512x16-ppc100-fp32"
METRIC = "particle-steps/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _workload(seed):
    from paper_1604_07713_gb300 import workloads as W
    cfg, mesh, parts = W.ccp(seed=seed, precision=W.FP32)
    cfg["mg_rel_tol"] = 1e-8
    return cfg, mesh, parts


def _config_json(ws):
    return {"workload": WORKLOAD, "cells": "512x16 uniform quadtree leaves", "particles_per_species": 819200,
            "species": 2, "precision": "fp32 particle state, fp64 Poisson residual",
            "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"replicas x{ws}",
            "poisson_rel_tol": 1e-8}


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.out = ""

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# oracle (CPU baseline and reference arm)
# ---------------------------------------------------------------------------------------
def _oracle_sim(seed):
    import oracle as O
    cfg, mesh, parts = _workload(seed)
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], 0, cfg["bc_x"], cfg["bc_y"])
    sim = O.Sim(cfg, M)
    for s in sorted(parts):
        sim.load(s, **parts[s])
    return sim


def _oracle_rate(sim, steps):
    tot, t = 0, 0.0
    for _ in range(steps):
        n = sum(sp.n for sp in sim.species)
        t0 = time.perf_counter()
        sim.step(1)
        t += time.perf_counter() - t0
        tot += n
    return tot / t, t


def cpu_baseline(seed, steps=12):
    sim = _oracle_sim(seed)
    sim.step(1)  # warm-up (imports, first solve)
    rate, t = _oracle_rate(sim, steps)
    return {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of the full workload (2 x 819,200 particles), FP64 oracle, "
                      f"single thread, {t:.1f} s"}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    sim = _oracle_sim(args.seed)
    for _ in range(args.warmup):
        sim.step(1)
    rate, t = _oracle_rate(sim, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_json(1),
            "cpu_baseline": {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps of the full workload after {args.warmup} warm-up, single thread"},
            "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def _traffic_record():
    """DRAM traffic per launch of the move kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1604_07713_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    if rec.get("csrc_sha256") != h.hexdigest():
        return None
    return rec


def run_gpu(args):
    import torch
    import paper_1604_07713_gb300 as G

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    G.build()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    stream = torch.cuda.Stream()
    cfg, mesh, parts = _workload(args.seed + rank)
    ctx = G.Context(cfg, stream_handle=stream.cuda_stream)
    ctx.set_mesh_dict(mesh)
    for s in sorted(parts):
        ctx.load(s, **parts[s])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        ctx.step(1)
    torch.cuda.synchronize()

    # timed region
    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = G.pic_get_launch_count(ctx.ctx)
    G.pic_set_timing(ctx.ctx, True)
    t_total = 0.0
    particle_steps = 0
    mover_particles = 0
    for _ in range(args.steps):
        c = ctx.counts()
        n = c["n_e"] + c["n_i"]
        with torch.cuda.stream(stream):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        ctx.step(1)
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        t_total += a.elapsed_time(b) * 1e-3
        particle_steps += n
        mover_particles += n
    torch.cuda.synchronize()
    phases = G.pic_get_timing(ctx.ctx)
    G.pic_set_timing(ctx.ctx, False)
    launches = G.pic_get_launch_count(ctx.ctx) - launches0
    clocks = sampler.stop()
    t_max = t_total
    if ws > 1:
        tt = torch.tensor([t_total], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
        ps = torch.tensor([float(particle_steps)], device="cuda")
        torch.distributed.all_reduce(ps)
        particle_steps_all = float(ps.item())
    else:
        particle_steps_all = float(particle_steps)
    value = particle_steps_all / t_max

    # roofline of the move pass (k_push in move mode, both species): algorithmic bytes per
    # particle = 28 B record read + 28 B record written; per leaf 32 B corner field + 8 B
    # list offsets (old and new), summed over the steps' particles
    nl = 512 * 16
    move_ms, move_launches = phases["move"]
    move_s = move_ms * 1e-3
    alg_bytes = 56.0 * mover_particles + args.steps * 2 * nl * (32 + 8)
    achieved = alg_bytes / move_s / 1e9 if move_s > 0 else 0.0
    tr = _traffic_record()
    roofline = {"bound": "hbm", "kernel": "k_push<float> (move pass, both species)", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": tr["move_bytes_per_step"] if tr else None,
                "peak_source": f"{peak_src} hbm_gbs", "alg_bytes_per_particle": 56,
                "launch_share": {k: round(v[0] / max(1e-9, sum(x[0] for x in phases.values())), 4)
                                 for k, v in phases.items() if v[1]}}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config_json(ws), "roofline": roofline, "clocks": clocks, "gpu_launches": int(launches),
            "phase_ms_per_step": {k: v[0] / args.steps for k, v in phases.items() if v[1]}}

    # end to end through the C ABI with host buffers: load (H2D) + one step + read phi (D2H)
    if not args.no_e2e:
        host = {s: {k: np.ascontiguousarray(v) for k, v in parts[s].items()} for s in parts}
        h2d = sum(v.nbytes for s in host for v in host[s].values())
        e2e_steps = max(3, min(args.steps, 10))
        t_e2e = 0.0
        n_e2e = 0
        for k in range(e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in sorted(host):
                ctx.load(s, **host[s])
            ctx.step(1)
            phi = ctx.fields(G.PIC_FIELD_PHI)
            t1 = time.perf_counter()
            if k > 0:
                t_e2e += t1 - t0
                n_e2e += sum(host[s]["x"].size for s in host)
        line["e2e"] = {"value": n_e2e / t_e2e, "unit": METRIC, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(phi.nbytes)}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.seed, steps=args.cpu_steps)
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gbpic", choices=["gbpic", "reference"])
    ap.add_argument("--seed", type=int, default=160407713)
    ap.add_argument("--cpu-steps", type=int, default=12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
