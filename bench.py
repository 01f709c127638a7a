"""Benchmark of the PIC-MCC particle cycle on one GB300 (or N independent replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbpic|reference]

Workloads (FP32 particle state):
  streamer (default): the 2D streamer on an adaptive quadtree -- 1 cm box of 128 x 128 root
      boxes refined up to 4 levels on the device, 5e7 electrons + ions in a channel, 3 MV/m
      background field, ionization MCC, split/merge toward 32 per leaf (band 8-128) and mesh
      adaptation every 10 steps inside the timed region.  State >> L2.
  ccp: the 2D capacitively coupled discharge (512 x 16 square cells, plates at x = 0 with
      200 V at 13.56 MHz and x = 6.7 cm grounded, periodic in y, electrons and 4 amu ions,
      100 macro-particles per cell and species = 2 x 819,200, dt = 1/(400 f)); L2 is flushed
      (256 MiB write) before every timed step, outside the timed events.
One step is the whole cycle: NGP deposit, multigrid Poisson, corner field, fused
gather/push/locate/MCC, cell-list update (plus the adaptation cadence).  Inputs are resident
in HBM when the timed region starts.

Prints one JSON line: particle-steps/s (whole job), the roofline of the dominant particle
kernel (the move pass of the fused push), the oracle's CPU baseline on a bounded sample,
the end-to-end rate through the C ABI with host buffers, clocks and kernel launches.
`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
WORKLOADS = ("ccp", "streamer", "ensemble", "ccp_implicit")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


PRECISION = {"fp32": 0, "fp64": 1}


def _workload(seed, name="ccp", n_particles=50_000_000, precision="fp32"):
    """The workload's config, mesh and particles; a name ending in '_implicit' selects the
    direct implicit scheme (§3 DIPIC) on the same inputs."""
    from paper_1604_07713_gb300 import workloads as W
    implicit = name.endswith("_implicit")
    base = name[:-len("_implicit")] if implicit else name
    if base == "streamer":
        cfg, mesh, parts = W.streamer_snapshot(n_particles=n_particles, seed=seed, precision=PRECISION[precision])
    else:
        cfg, mesh, parts = W.ccp(seed=seed, precision=PRECISION[precision])
        cfg["mg_rel_tol"] = 1e-8
    cfg["implicit"] = 1 if implicit else 0
    return cfg, mesh, parts


def _config_json(ws, name="ccp", extra=None, precision="fp32"):
    implicit = name.endswith("_implicit")
    name = name[:-len("_implicit")] if implicit else name
    if name == "ensemble":
        d = {"workload": "ccp-ensemble-256-fp32", "instances": 256,
             "cells": "per instance 64-512 x 16 uniform leaves (multiples of 16 in x)",
             "species": 2, "precision": "fp32 particle state, fp64 Poisson residual",
             "batching": "all instances in one context; one launch solves every instance's Poisson",
             "l2": "inputs larger than L2 (particle state >> 129 MB)",
             "parallelism": "one rank" if ws == 1 else f"the 256 instances split over {ws} ranks by particle count (LPT)",
             "poisson_rel_tol": 1e-8}
    elif name == "streamer":
        d = {"workload": f"streamer-amr-128x128-l4-{precision}", "cells": "adaptive quadtree, 128x128 roots, up to 4 levels",
             "species": 2, "precision": "fp32 particle state, fp64 Poisson residual",
             "adapt": "pic_adapt (mesh + split/merge) every 10 steps inside the timed region",
             "l2": "inputs larger than L2 (particle state >> 129 MB)", "parallelism": f"replicas x{ws}",
             "poisson_rel_tol": 1e-8}
    else:
        d = {"workload": f"ccp-512x16-ppc100-{precision}", "cells": "512x16 uniform quadtree leaves", "particles_per_species": 819200,
             "species": 2, "precision": "fp32 particle state, fp64 Poisson residual",
             "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"replicas x{ws}",
             "poisson_rel_tol": 1e-8}
    if implicit:
        d["workload"] += "-implicit"
        d["scheme"] = ("direct implicit (§3 DIPIC): predictor push, Poisson with the susceptibility "
                       "1 + (omega_p dt)^2, corrector push")
    if extra:
        d.update(extra)
    return d


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
ORACLE_STREAMER_PARTICLES = 200_000


ORACLE_ENSEMBLE_INSTANCES = 2


def _oracle_sims_ensemble(seed):
    import oracle as O
    from paper_1604_07713_gb300 import workloads as W
    sims = []
    for cfg, mesh, factory, _ in W.ensemble(256, seed=seed)[:ORACLE_ENSEMBLE_INSTANCES]:
        M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], 0, cfg["bc_x"], cfg["bc_y"])
        sim = O.Sim(cfg, M)
        parts = factory()
        for s_ in sorted(parts):
            sim.load(s_, **parts[s_])
        sims.append(sim)
    return sims


def _oracle_sim(seed, name="ccp"):
    import oracle as O
    if name == "streamer":
        cfg, mesh, parts = _workload(seed, "streamer", ORACLE_STREAMER_PARTICLES)
        M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], mesh["lmax"], cfg["bc_x"], cfg["bc_y"])
        sim = O.Sim(cfg, M)
        for s in sorted(parts):
            sim.load(s, **parts[s])
        for _ in range(mesh["lmax"] + 1):  # refine the uniform roots onto the particles
            sim.fields()
            sim.adapt(mesh=True, particles=False)
        sim.fields()
        sim.adapt()
        return sim
    cfg, mesh, parts = _workload(seed, name)
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], 0, cfg["bc_x"], cfg["bc_y"])
    sim = O.Sim(cfg, M)
    for s in sorted(parts):
        sim.load(s, **parts[s])
    return sim


def _oracle_rate(sim, steps, adapt_every=0):
    tot, t = 0, 0.0
    for k in range(steps):
        n = sum(sp.n for sp in sim.species)
        t0 = time.perf_counter()
        sim.step(1)
        if adapt_every and (k + 1) % adapt_every == 0:
            sim.adapt()
        t += time.perf_counter() - t0
        tot += n
    return tot / t, t


def _sample_text(name, steps, t):
    if name == "streamer":
        return (f"{steps} steps (adaptation every 10) of the streamer workload at {ORACLE_STREAMER_PARTICLES:,} "
                f"particles (the GPU runs 5e7) on a mesh the oracle adapted itself, FP64, one thread, {t:.1f} s")
    return f"{steps} steps of the full workload (2 x 819,200 particles), FP64 oracle, one thread, {t:.1f} s"


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_worker(seed, name, steps, barrier, queue):
    """One core's share of the all-core baseline: its own bounded sample, timed after every
    worker has finished its setup."""
    sim = _oracle_sim(seed, name)
    sim.step(1)
    barrier.wait()
    queue.put(_oracle_rate(sim, steps, 10 if name == "streamer" else 0))


def cpu_baseline_all_cores(seed, steps, name):
    """The oracle as it stands (one thread per process) on every host core at once: one
    independent bounded sample per core (seeds seed + k), started together; the job's rate is
    the sum of the processes' rates.  Processes are spawned, never forked after CUDA use."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(seed + k, name, steps, barrier, queue)) for k in range(n)]
    for p in procs:
        p.start()
    res = [queue.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    return sum(r for r, _ in res), max(t for _, t in res), n


def cpu_baseline(seed, steps=12, name="ccp"):
    if name == "ensemble":
        sims = _oracle_sims_ensemble(seed)
        tot, t = 0, 0.0
        for sim in sims:
            sim.step(1)
            r, tt = _oracle_rate(sim, max(1, steps // len(sims)))
            tot += r * tt
            t += tt
        return {"value": tot / t, "unit": METRIC, "cores": 1, "kind": "oracle",
                "sample": f"the first {len(sims)} of the 256 instances, {max(1, steps // len(sims))} steps each, "
                          f"FP64 oracle, single thread, {t:.1f} s"}
    sim = _oracle_sim(seed, name)
    sim.step(1)  # warm-up (imports, first solve)
    rate, t = _oracle_rate(sim, steps, 10 if name == "streamer" else 0)
    del sim
    single = {"value": rate, "cores": 1, "sample": _sample_text(name, steps, t)}
    try:
        rate_all, t_all, n = cpu_baseline_all_cores(seed, steps, name)
    except Exception as e:  # the single-thread figure stands alone
        return {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle", "cpu_model": _cpu_model(),
                "sample": _sample_text(name, steps, t), "all_cores_error": str(e)[:200]}
    return {"value": rate_all, "unit": METRIC, "cores": n, "kind": "oracle", "cpu_model": _cpu_model(),
            "nproc": n, "sample": f"{n} processes at once, each: " + _sample_text(name, steps, t_all),
            "single_thread": single}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    if args.workload == "ensemble":
        base = cpu_baseline(args.seed, steps=args.steps * ORACLE_ENSEMBLE_INSTANCES, name="ensemble")
        rate = base["value"]
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": _config_json(1, "ensemble"), "cpu_baseline": base,
                "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    # every host core runs its own bounded sample of the workload (warm-up steps included in
    # each process's setup), started together; the rate is the sum over the processes
    rate, t, n = cpu_baseline_all_cores(args.seed, args.steps, args.workload)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config_json(1, args.workload, precision=args.precision),
            "cpu_baseline": {"value": rate, "unit": METRIC, "cores": n, "kind": "oracle", "cpu_model": _cpu_model(),
                             "sample": f"{n} processes at once, each: " + _sample_text(args.workload, args.steps, t)},
            "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
# The push kernel's translation unit: the sources that decide its code and so its DRAM
# traffic (the kernel file, the internal header it includes and the ABI header).
PUSH_SOURCES = ("paper_1604_07713_gb300/csrc/pic_particles.cu", "paper_1604_07713_gb300/csrc/pic_internal.cuh",
                "include/gbpic.h")


def _csrc_hash():
    h = hashlib.sha256()
    for f in PUSH_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def _traffic_record(name):
    """DRAM bytes per launch of the move kernel from the committed ncu summary, if that was
    taken on the push kernel's current sources (PUSH_SOURCES) and this workload (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(name)
    if not rec or rec.get("csrc_sha256") != _csrc_hash():
        return None
    return rec


def _aggregate(t_local, particle_steps_local, ws, device):
    """The whole job over ranks: the slowest rank's timed seconds and the particle-steps of
    all ranks (FP64 all-reduces on `device`; one rank: the local values)."""
    if ws <= 1:
        return float(t_local), float(particle_steps_local)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ps = torch.tensor([float(particle_steps_local)], dtype=torch.float64, device=device)
    dist.all_reduce(ps)
    return float(tt.item()), float(ps.item())


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
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    name = args.workload
    streamer = name == "streamer"

    stream = torch.cuda.Stream()
    ensemble = name == "ensemble"
    if ensemble:
        from paper_1604_07713_gb300 import workloads as W
        from paper_1604_07713_gb300.shard import lpt_shard
        members = W.ensemble(256, seed=args.seed)
        if ws > 1:  # the same 256 instances, split over the ranks by particle count (LPT)
            mine = lpt_shard([m[3] for m in members], ws)[rank]
            members = [members[i] for i in mine]
        cfg = members[0][0]
        ctx = G.Context([m[0] for m in members], stream_handle=stream.cuda_stream)
        for i, (c_i, mesh_i, factory, _) in enumerate(members):
            ctx.set_mesh_dict(mesh_i, inst=i)
            parts_i = factory()
            for s_ in sorted(parts_i):
                ctx.load(s_, **parts_i[s_], inst=i)
        n_inst = len(members)
        mesh, parts = members[0][1], None
    else:
        cfg, mesh, parts = _workload(args.seed + rank, name, args.particles, args.precision)
        ctx = G.Context(cfg, stream_handle=stream.cuda_stream)
        ctx.set_mesh_dict(mesh)
        for s in sorted(parts):
            ctx.load(s, **parts[s])
        n_inst = 1
    if streamer:  # refine the uniform roots onto the particles, then manage them (setup, untimed)
        for _ in range(mesh["lmax"] + 1):
            ctx.compute_fields(allow_notconv=True)
            ctx.adapt(G.PIC_ADAPT_MESH)
        ctx.compute_fields(allow_notconv=True)
        ctx.adapt()

    def counts_all():
        tot = {"n_e": 0, "n_i": 0, "n_leaves": 0, "mg_cycles": 0}
        for i in range(n_inst):
            c = ctx.counts(i)
            for k in tot:
                tot[k] += c[k]
        return tot
    flush = None if (streamer or ensemble) else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    adapt_every = cfg.get("adapt_every", 0) if streamer else 0

    def one_step(k):
        ctx.step(1)
        if adapt_every and (k + 1) % adapt_every == 0:
            ctx.adapt()

    # launch shapes chosen by the library's autotuner (setup, untimed: its steps are ordinary
    # steps under candidate shapes, and no result depends on the shape)
    tuned_steps = ctx.autotune(args.autotune_steps, allow_notconv=True) if args.autotune_steps > 0 else 0
    tuning = dict(ctx.tuning(), steps=tuned_steps)
    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()

    # timed region
    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    G.pic_set_timing(ctx.ctx, True)
    t_total = 0.0
    particle_steps = 0
    leaf_steps = 0
    launches = 0  # the library's launches inside the timed steps (not the count read-outs between them)
    for k in range(args.steps):
        c = counts_all()
        n = c["n_e"] + c["n_i"]
        with torch.cuda.stream(stream):
            if flush is not None:
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        l0 = G.pic_get_launch_count(ctx.ctx)
        one_step(args.warmup + k)
        launches += G.pic_get_launch_count(ctx.ctx) - l0
        with torch.cuda.stream(stream):
            b.record(stream)
        b.synchronize()
        t_total += a.elapsed_time(b) * 1e-3
        particle_steps += n
        leaf_steps += c["n_leaves"]
    torch.cuda.synchronize()
    phases = G.pic_get_timing(ctx.ctx)
    G.pic_set_timing(ctx.ctx, False)
    clocks = sampler.stop()
    t_max, particle_steps_all = _aggregate(t_total, particle_steps, ws, "cuda")
    value = particle_steps_all / t_max
    final = counts_all()

    # Roofline of the fused push (k_push, both species, lists updated in place): algorithmic
    # bytes = the record (u, v, vx, vy, vz, w in the state precision, id u32) read once and its
    # five changed words (u, v, vx, vy, vz) written once per particle -- 11 rs + 4 bytes --
    # plus per leaf and species the 8 corner field values, the list bounds (start, end) and
    # the staying count and weight sum written.  The extra words of records that change slot
    # (w, id, order key) are not counted.
    rs = 8 if args.precision == "fp64" else 4
    move_ms, move_launches = phases["move"]
    push_label = f"k_push<{'double' if rs == 8 else 'float'}> in-place push (both species)"
    if name.endswith("_implicit"):
        push_label += ", the implicit scheme's predictor and corrector passes"
    graph_ms = phases.get("graph", (0.0, 0))[0]
    if ensemble and move_ms > 0.0 and graph_ms > 0.0:
        # the batched step's replays time their phases inside the graph (event nodes)
        push_label = f"k_push_batch<{'double' if rs == 8 else 'float'}> (every instance, both species)"
    if move_ms == 0.0 and graph_ms > 0.0:
        # an ensemble replays whole steps as one graph: the push cannot be timed alone, so the
        # whole step's time stands in (a lower bound of the push's fraction)
        move_ms = phases["graph"][0]
        push_label = "whole step (graph replay; push bytes over step time: a lower bound)"
    move_s = move_ms * 1e-3
    passes = 2 if name.endswith("_implicit") else 1  # the implicit scheme's predictor and corrector
    alg_bytes = passes * ((11 * rs + 4) * particle_steps + leaf_steps * 2 * (10 * rs + 12))
    achieved = alg_bytes / move_s / 1e9 if move_s > 0 else 0.0
    tr = _traffic_record(name) if args.precision == "fp32" else None
    # with phases timed inside graph replays, the replay's total is not a phase of its own
    inner = graph_ms > 0.0 and any(v[0] > 0.0 for k, v in phases.items() if k != "graph")
    tot_ms = sum(v[0] for k, v in phases.items() if not (inner and k == "graph"))
    roofline = {"bound": "hbm", "kernel": push_label,
                "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": tr["move_dram_bytes_per_step"] if tr else None,
                "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                "alg_bytes_per_step": alg_bytes / args.steps,
                "phase_share": {k: round(v[0] / max(1e-9, tot_ms), 4) for k, v in phases.items()
                                if v[1] and not (inner and k == "graph")}}
    # The whole particle cycle (deposit, corner field, list preparation, push, scans and list
    # repairs, per-leaf sorts): the push's algorithmic bytes plus the corner field written and
    # the deposit's per-leaf charge, over the summed CUDA-event time of those phases.  Records
    # that change leaf are written to free slots and sorted into place, traffic that is not
    # counted here, so this fraction is a lower bound.
    cycle_phases = ("deposit", "node_e", "lists", "scan", "move", "sort")
    cycle_ms = sum(phases[k][0] for k in cycle_phases if k in phases)
    cycle_bytes = alg_bytes + leaf_steps * (8 * rs + 8)
    if cycle_ms > 0.0 and (graph_ms == 0.0 or inner):
        ca = cycle_bytes / (cycle_ms * 1e-3) / 1e9
        roofline["particle_cycle"] = {"achieved": ca, "frac": ca / hbm_peak, "unit": "GB/s",
                                      "phases": list(cycle_phases), "ms_per_step": cycle_ms / args.steps,
                                      "alg_bytes_per_step": cycle_bytes / args.steps}
    list_stats = [G.pic_get_list_stats(ctx.ctx, 0, s_) for s_ in range(cfg["n_species"])]
    extra = {"precision": f"{args.precision} particle state and push, fp64 Poisson residual",
             "list_relayouts_since_load": [r for r, _, _ in list_stats],
             "list_tail_moves_since_load": [m for _, m, _ in list_stats],
             "particles_mean": int(particle_steps / args.steps),
             "particles_end": int(final["n_e"] + final["n_i"]), "leaves_end": int(final["n_leaves"]),
             "poisson_cycles_last": int(final["mg_cycles"]), "autotune": tuning}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if ensemble and ws > 1 else "weak", "vs_baseline": None,
            "dtype": "f64" if rs == 8 else "f32", "data": "synthetic",
            "config": _config_json(ws, name, extra, args.precision), "roofline": roofline, "clocks": clocks,
            "gpu_launches": int(launches),
            "phase_ms_per_step": {k: round(v[0] / args.steps, 5) for k, v in phases.items() if v[1]}}

    if ensemble and args.sequential > 0:
        # the same instances advanced one after another, each in its own context
        t_seq, ps_seq = 0.0, 0
        for c_i, mesh_i, factory, _ in members[:args.sequential]:
            with G.Context(c_i, stream_handle=stream.cuda_stream) as one:
                one.set_mesh_dict(mesh_i)
                parts_i = factory()
                for s_ in sorted(parts_i):
                    one.load(s_, **parts_i[s_])
                one.step(args.warmup)
                c0 = one.counts()
                torch.cuda.synchronize()
                with torch.cuda.stream(stream):
                    a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                one.step(args.steps)
                with torch.cuda.stream(stream):
                    b.record(stream)
                b.synchronize()
                t_seq += a.elapsed_time(b) * 1e-3
                ps_seq += (c0["n_e"] + c0["n_i"]) * args.steps
        line["sequential_single_instance"] = {"value": ps_seq / t_seq, "unit": METRIC,
                                              "instances": args.sequential,
                                              "note": "the first instances of the ensemble, each alone, same steps"}
    # end to end through the C ABI with host buffers: load (H2D) + one step + read phi (D2H)
    if not args.no_e2e and not ensemble:
        # the step's inputs in pinned host memory (numpy views of page-locked tensors)
        host = {s: {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy() for k, v in parts[s].items()}
                for s in parts}
        h2d = sum(v.nbytes for s in host for v in host[s].values())
        e2e_steps = 6 if streamer else max(3, min(args.steps, 10))
        t_e2e = 0.0
        n_e2e = 0
        iter_ms = []
        e2e_warm = 3  # untimed, like the device-timed steps' warm-up (the first reloads re-size the buffers)
        for k in range(e2e_warm + e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in sorted(host):
                ctx.load(s, **host[s])
            ctx.step(1)
            phi = ctx.fields(G.PIC_FIELD_PHI)
            t1 = time.perf_counter()
            if k >= e2e_warm:
                t_e2e += t1 - t0
                n_e2e += sum(host[s]["x"].size for s in host)
                iter_ms.append(round((t1 - t0) * 1e3, 3))
        line["e2e"] = {"value": n_e2e / t_e2e, "unit": METRIC, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(phi.nbytes), "iter_ms": iter_ms}
    ctx.close()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.seed, steps=args.cpu_steps, name=name)
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
    ap.add_argument("--workload", default="streamer", choices=WORKLOADS)
    ap.add_argument("--particles", type=int, default=50_000_000, help="streamer workload: total particles")
    ap.add_argument("--precision", default="fp32", choices=tuple(PRECISION),
                    help="particle state and push arithmetic (ccp and streamer workloads)")
    ap.add_argument("--sequential", type=int, default=0,
                    help="ensemble workload: also time this many instances one after another")
    ap.add_argument("--cpu-steps", type=int, default=12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--autotune-steps", type=int, default=20,
                    help="steps the launch-shape autotuner may run during setup (0: default shapes)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
