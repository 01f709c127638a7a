"""Precision study of the streamer (FP32 cell-relative push and compensated deposit, FP32
multigrid smoothing with FP64 residual and refinement to 1e-10 relative residual).

Run on a GPU: ``python tests/precision_study.py [--subset 1000000] [--particles 50000000]``.
Prints one JSON line:

- ``subset_vs_fp64_oracle``: a streamer snapshot of ``--subset`` particles, adapted by the
  oracle; the FP32 and FP64 GPU paths start from that mesh and population.  Errors of phi,
  the corner field E and rho (relative L2 over leaves), and of the per-leaf electron and ion
  counts after one step, against the oracle.
- ``full_fp32_vs_fp64_gpu``: the full-size snapshot, adapted by the FP32 path, read back and
  loaded into an FP64 context; the same errors of FP32 against FP64 on the GPU.  A particle
  whose offset in its leaf is exactly 0 lies on the face it shares with the leaf below; the
  read-back position x = (corner + offset * side) * h can round below the face, so it is
  moved up by one unit in the last place before the FP64 context locates it in its leaf.

Not collected by pytest (a script); it is the measurement behind the precision table of the
design notes.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), os.pardir))

import oracle as O  # noqa: E402
import paper_1604_07713_gb300 as G  # noqa: E402
from paper_1604_07713_gb300 import workloads as W  # noqa: E402


def rel(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(np.asarray(a, dtype=float) - b)) / (nb if nb > 0 else 1.0)


def fields(ctx):
    return {"rho": ctx.fields(G.PIC_FIELD_RHO), "phi": ctx.fields(G.PIC_FIELD_PHI),
            "E": ctx.fields(G.PIC_FIELD_NODE_E).reshape(-1)}


def errors(f, g, ca, cb):
    return {"phi": rel(f["phi"], g["phi"]), "E": rel(f["E"], g["E"]), "rho": rel(f["rho"], g["rho"]),
            "n_e_after_step": rel(ca[0], cb[0]), "n_i_after_step": rel(ca[1], cb[1])}


def leaf_corners(nx0, lmax, root, morton, level):
    """Lower-left corner of every leaf on the finest lattice (root box, then Morton bits)."""
    root = root.astype(np.int64); morton = morton.astype(np.int64); level = level.astype(np.int64)
    mx = np.zeros_like(morton); my = np.zeros_like(morton)
    for b in range(16):
        mx |= ((morton >> (2 * b)) & 1) << b
        my |= ((morton >> (2 * b + 1)) & 1) << b
    ix = ((root % nx0) << lmax) + (mx << (lmax - level))
    iy = ((root // nx0) << lmax) + (my << (lmax - level))
    return ix, iy


def on_own_leaf(p, corners, hf):
    """Positions that locate in the leaf they were read from (see the module note)."""
    leaf = p["leaf"].astype(np.int64)
    x, y = p["x"].copy(), p["y"].copy()
    for arr, lo in ((x, corners[0]), (y, corners[1])):
        low = np.floor(arr / hf) < lo[leaf]
        arr[low] = np.nextafter(arr[low], np.inf)
    return x, y


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--subset", type=int, default=1_000_000)
    ap.add_argument("--particles", type=int, default=50_000_000)
    ap.add_argument("--seed", type=int, default=160407713)
    args = ap.parse_args()
    G.build()
    O.build()
    t0 = time.perf_counter()
    out = {"study": "precision", "workload": "streamer-amr-128x128-l4", "poisson_rel_tol": 1e-10}
    # (1) subset against the FP64 oracle
    cfg, mesh, parts = W.streamer_snapshot(n_particles=args.subset, seed=args.seed, precision=W.FP64)
    cfg["mg_rel_tol"] = 1e-10
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], mesh["lmax"], cfg["bc_x"], cfg["bc_y"])
    sim = O.Sim(cfg, M)
    for s in sorted(parts):
        sim.load(s, **parts[s])
    for _ in range(mesh["lmax"] + 1):
        sim.fields()
        sim.adapt(mesh=True, particles=False)
    sim.fields()
    sim.adapt()
    Mo = sim.mesh
    mesh_o = dict(nx0=mesh["nx0"], ny0=mesh["ny0"], h0=mesh["h0"], root=Mo.root, level=Mo.level,
                  morton=Mo.morton)
    state = {s: dict(x=sp.x.copy(), y=sp.y.copy(), vx=sp.vx.copy(), vy=sp.vy.copy(), vz=sp.vz.copy(),
                     w=sp.w.copy(), ids=sp.id.astype(np.uint64)) for s, sp in enumerate(sim.species)}
    rho_o, phi_o, E_o = sim.fields()
    f_o = {"rho": rho_o, "phi": phi_o, "E": E_o.reshape(-1)}
    sim.step(1)
    cnt_o = [np.bincount(sp.leaf, minlength=Mo.nleaf).astype(float) for sp in sim.species]
    sub = {"particles": int(sum(v["x"].size for v in state.values())), "leaves": int(Mo.nleaf)}
    for name, prec in (("fp32", W.FP32), ("fp64", W.FP64)):
        with G.Context(dict(cfg, precision=prec)) as ctx:
            ctx.set_mesh_dict(mesh_o)
            for s in sorted(state):
                ctx.load(s, **state[s])
            ctx.compute_fields()
            f = fields(ctx)
            ctx.step(1)
            c = [ctx.fields(G.PIC_FIELD_COUNT_E), ctx.fields(G.PIC_FIELD_COUNT_I)]
        sub[name] = errors(f, f_o, c, cnt_o)
    out["subset_vs_fp64_oracle"] = sub
    # (2) full size: FP32 against FP64 on the GPU from one state
    cfg32, mesh32, parts32 = W.streamer_snapshot(n_particles=args.particles, seed=args.seed, precision=W.FP32)
    cfg32["mg_rel_tol"] = 1e-10
    with G.Context(cfg32) as a:
        a.set_mesh_dict(mesh32)
        for s in sorted(parts32):
            a.load(s, **parts32[s])
        del parts32
        for _ in range(mesh32["lmax"] + 1):
            a.compute_fields(allow_notconv=True)
            a.adapt(G.PIC_ADAPT_MESH)
        a.compute_fields(allow_notconv=True)
        a.adapt()
        r, m, lv = a.mesh()
        mesh_a = dict(nx0=mesh32["nx0"], ny0=mesh32["ny0"], h0=mesh32["h0"], root=r, morton=m, level=lv)
        corners = leaf_corners(mesh32["nx0"], mesh32["lmax"], r, m, lv)
        hf = mesh32["h0"] / (1 << mesh32["lmax"])
        with G.Context(dict(cfg32, precision=W.FP64)) as b:
            b.set_mesh_dict(mesh_a)
            n_full = 0
            for s in (0, 1):
                p = a.particles(s)
                x, y = on_own_leaf(p, corners, hf)
                b.load(s, x, y, p["vx"], p["vy"], p["vz"], p["w"], ids=p["id"])
                n_full += int(x.size)
                del p
            a.compute_fields()
            b.compute_fields()
            fa, fb = fields(a), fields(b)
            same = [bool(np.array_equal(a.fields(k), b.fields(k)))
                    for k in (G.PIC_FIELD_COUNT_E, G.PIC_FIELD_COUNT_I)]
            a.step(1)
            b.step(1)
            ca = [a.fields(G.PIC_FIELD_COUNT_E), a.fields(G.PIC_FIELD_COUNT_I)]
            cb = [b.fields(G.PIC_FIELD_COUNT_E), b.fields(G.PIC_FIELD_COUNT_I)]
    full = {"particles": n_full, "leaves": int(r.size), "same_leaf_counts_at_start": same}
    full.update(errors(fa, fb, ca, cb))
    out["full_fp32_vs_fp64_gpu"] = full
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out))


if __name__ == "__main__":
    main()
