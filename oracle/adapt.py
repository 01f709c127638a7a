"""ORACLE -- test infrastructure only.

Mesh adaptation and particle management of the cell-based AMR grid, restated from
Kolobov & Arslanbekov (arXiv:1604.07713):

* §3.1: when a coarse cell is refined its particles are stored in the new cells according to
  their position; when cells are coarsened their particles go to the new coarse cell.
* §4.3: the AMR grid as particle management for exponential electron/ion growth; particle
  splitting (one particle replaced by four in 2D) and merging.

The refinement criterion, the merge rule and the list orders are readings (the paper gives
none); they are written out in the functions below and followed identically by the CUDA path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np


def _lib():
    from . import _Mesh, lib
    L = lib()
    if not getattr(L, "_adapt_declared", False):
        L.or_adapt_balance.argtypes = [C.POINTER(_Mesh), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_adapt_balance.restype = C.c_int32
        L._adapt_declared = True
    return L


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def adapt_mesh(sim) -> dict:
    """Refine / coarsen the leaves of ``sim.mesh``; hand the particles and the potential over.

    Refine leaf l (level < max_level) if its electron count exceeds refine_count or its
    centre |E| exceeds refine_field * e_ref.  A quartet of sibling leaves coarsens when none
    of them refines, their electron counts sum to at most coarsen_count and every |E| is
    below coarsen_field * e_ref.  Then 2:1 balance across faces and corners (refinement wins).
    Particle lists: stable by new leaf over the old list order (refined leaves hand each child
    the particles inside it, in order; a coarsened quartet's list is the four lists in child
    order).  Potential: children take the parent's value, a parent the mean of its children.
    """
    from . import Mesh
    M = sim.mesh
    cfg = sim.cfg
    n = M.nleaf
    level = M.level.astype(np.int32)
    cnt = sim.counts(0).astype(np.int64)
    walls = getattr(sim, "last_walls", None)
    if walls is None:
        walls = sim.walls()
    emag = M.cell_emag(sim.phi, walls)
    e_ref = cfg.get("e_ref", 1.0)
    refine = ((level < M.lmax) & ((cnt > cfg.get("refine_count", 128)) |
                                  (emag > cfg.get("refine_field", 1.5) * e_ref))).astype(np.int32)
    # sibling quartets: 4 consecutive leaves of one parent
    group = np.full(n, -1, np.int64)
    gactive = np.zeros(n, np.int32)
    i = 0
    while i + 3 < n:
        if (level[i] >= 1 and (M.morton[i] & 3) == 0 and np.all(level[i:i + 4] == level[i])
                and np.all(M.root[i:i + 4] == M.root[i])
                and np.all((M.morton[i:i + 4] >> 2) == (M.morton[i] >> 2))):
            group[i:i + 4] = i
            ok = (not refine[i:i + 4].any() and cnt[i:i + 4].sum() <= cfg.get("coarsen_count", 32)
                  and np.all(emag[i:i + 4] < cfg.get("coarsen_field", 1.2) * e_ref))
            gactive[i] = 1 if ok else 0
            i += 4
        else:
            i += 1
    sweeps = _lib().or_adapt_balance(C.byref(M._c), _p(level), _p(refine), _p(group), _p(gactive))
    # new leaf list in Morton order
    roots, levels, mortons, new_of = [], [], [], np.empty(n, np.int64)
    k = 0
    for i in range(n):
        g = group[i]
        if g >= 0 and gactive[g]:
            if i == g:
                roots.append(M.root[i]); levels.append(level[i] - 1); mortons.append(M.morton[i] >> 2)
                k += 1
            new_of[i] = k - 1
        elif refine[i]:
            for c in range(4):
                roots.append(M.root[i]); levels.append(level[i] + 1); mortons.append((int(M.morton[i]) << 2) | c)
            new_of[i] = k
            k += 4
        else:
            roots.append(M.root[i]); levels.append(level[i]); mortons.append(M.morton[i])
            new_of[i] = k
            k += 1
    M2 = Mesh(M.nx0, M.ny0, M.h0, M.lmax, M.bc_x, M.bc_y, np.array(roots, np.int32),
              np.array(levels, np.int32), np.array(mortons, np.uint32))
    # potential carried over
    phi2 = np.empty(M2.nleaf)
    for i in range(n):
        g = group[i]
        if g >= 0 and gactive[g]:
            if i == g:
                phi2[new_of[i]] = np.mean(sim.phi[i:i + 4])
        elif refine[i]:
            phi2[new_of[i]:new_of[i] + 4] = sim.phi[i]
        else:
            phi2[new_of[i]] = sim.phi[i]
    # particles: new leaf by position, stable over the old list order
    for s, sp in enumerate(sim.species):
        if sp is None or sp.n == 0:
            continue
        nl = M2.locate(sp.x, sp.y)
        order = np.argsort(nl, kind="stable")
        sp2 = sp.take(order)
        sp2.leaf = nl[order]
        sim.species[s] = sp2
    sim.mesh = M2
    sim.phi = phi2
    return dict(refined=int(refine.sum()), coarsened=int(gactive.sum()), sweeps=int(sweeps),
                n_leaves=M2.nleaf)


# ---------------------------------------------------------------------------------------
# Split / merge (§4.3)
# ---------------------------------------------------------------------------------------
def _split_once(u, v, w, vel, ids):
    """One particle -> four of weight w/4 at (u -+ d, v -+ d), d = min(0.25 * distance to the
    nearest leaf face, 2^-10) in leaf units; velocity kept; order (-,-), (+,-), (-,+), (+,+).
    Charge, mass, momentum, energy and the charge centre are conserved exactly."""
    d = min(0.25 * min(u, 1.0 - u, v, 1.0 - v), 2.0 ** -10)
    out = []
    for k, (sx, sy) in enumerate(((-1, -1), (1, -1), (-1, 1), (1, 1))):
        out.append((u + sx * d, v + sy * d, w / 4.0, vel, ids if k == 0 else None))
    return out


def _energy_bins(vx, vy, vz, half_m, fp32):
    """16 energy bins over the leaf's range, decided in the particle state's precision."""
    if fp32:
        f = np.float32
        vx, vy, vz = vx.astype(f), vy.astype(f), vz.astype(f)
        eps = f(half_m) * ((vx * vx + vy * vy) + vz * vz)
        lo, hi = eps.min(), eps.max()
        rng = f(hi - lo)
        if rng == f(0):
            return np.zeros(eps.size, np.int64)
        q = ((eps - lo) * f(16)) / rng
        return np.clip(np.floor(q).astype(np.int64), 0, 15)
    eps = half_m * ((vx * vx + vy * vy) + vz * vz)
    lo, hi = eps.min(), eps.max()
    rng = hi - lo
    if rng == 0:
        return np.zeros(eps.size, np.int64)
    q = ((eps - lo) * 16.0) / rng
    return np.clip(np.floor(q).astype(np.int64), 0, 15)


def split_merge(sim) -> dict:
    """Per leaf and species, with c particles (cfg ppc_min, ppc_max, ppc_target):

    * 0 < c < ppc_min: split every particle 1 -> 4 (recursively r times, the least r with
      c 4^r >= ppc_min), children in depth-first order; the first child keeps the parent id,
      the others take new ids in list order.
    * c > ppc_max: order the list by (energy bin, id) and cut it into ppc_target consecutive
      groups, the first (c mod ppc_target) of size ceil(c / ppc_target), the rest floor; each
      group becomes one particle with the summed weight, the weighted mean position and
      velocity and the smallest id (charge, mass and momentum conserved; kinetic energy drops
      by the groups' internal spread).  With c <= 2 ppc_target this merges consecutive pairs
      and keeps the rest.
    * otherwise the list is unchanged.
    """
    cfg = sim.cfg
    M = sim.mesh
    lo, hi, tgt = cfg.get("ppc_min", 8), cfg.get("ppc_max", 128), cfg.get("ppc_target", 32)
    fp32 = cfg.get("precision", 0) == 0
    stats = dict(split=0, merged=0, new_ids=0)
    hf = M.hf
    for s, sp in enumerate(sim.species):
        if sp is None or sp.n == 0:
            continue
        starts = np.searchsorted(sp.leaf, np.arange(M.nleaf + 1))
        cols = {k: [] for k in ("x", "y", "vx", "vy", "vz", "w", "id", "leaf")}
        for l in range(M.nleaf):
            a, b = starts[l], starts[l + 1]
            c = b - a
            if c == 0:
                continue
            h = M.s[l] * hf
            x0, y0 = M.ix[l] * hf, M.iy[l] * hf
            if c < lo:
                r = 0
                while c * 4 ** r < lo:
                    r += 1
                for p in range(a, b):
                    parts = [((sp.x[p] - x0) / h, (sp.y[p] - y0) / h, sp.w[p],
                              (sp.vx[p], sp.vy[p], sp.vz[p]), sp.id[p])]
                    for _ in range(r):
                        nxt = []
                        for (u, v, w, vel, pid) in parts:
                            nxt.extend(_split_once(u, v, w, vel, pid))
                        parts = nxt
                    for (u, v, w, vel, pid) in parts:
                        if pid is None:
                            pid = sim.next_id
                            sim.next_id += 1
                            stats["new_ids"] += 1
                        cols["x"].append(x0 + u * h); cols["y"].append(y0 + v * h)
                        cols["vx"].append(vel[0]); cols["vy"].append(vel[1]); cols["vz"].append(vel[2])
                        cols["w"].append(w); cols["id"].append(pid); cols["leaf"].append(l)
                stats["split"] += c
            elif c > hi:
                bins = _energy_bins(sp.vx[a:b], sp.vy[a:b], sp.vz[a:b], 0.5 * sp.m, fp32)
                order = np.lexsort((sp.id[a:b], bins)) + a
                q, rem = divmod(c, tgt)
                pos = 0
                for g in range(tgt):
                    size = q + 1 if g < rem else q
                    idx = order[pos:pos + size]
                    pos += size
                    W = 0.0; X = 0.0; Y = 0.0; VX = 0.0; VY = 0.0; VZ = 0.0
                    for p in idx:
                        W += sp.w[p]
                    for p in idx:
                        X += sp.w[p] * sp.x[p]; Y += sp.w[p] * sp.y[p]
                        VX += sp.w[p] * sp.vx[p]; VY += sp.w[p] * sp.vy[p]; VZ += sp.w[p] * sp.vz[p]
                    cols["x"].append(X / W); cols["y"].append(Y / W)
                    cols["vx"].append(VX / W); cols["vy"].append(VY / W); cols["vz"].append(VZ / W)
                    cols["w"].append(W); cols["id"].append(int(sp.id[idx].min())); cols["leaf"].append(l)
                stats["merged"] += c - tgt
            else:
                for p in range(a, b):
                    cols["x"].append(sp.x[p]); cols["y"].append(sp.y[p])
                    cols["vx"].append(sp.vx[p]); cols["vy"].append(sp.vy[p]); cols["vz"].append(sp.vz[p])
                    cols["w"].append(sp.w[p]); cols["id"].append(sp.id[p]); cols["leaf"].append(l)
        from . import Species
        sim.species[s] = Species(sp.q, sp.m, np.array(cols["x"]), np.array(cols["y"]), np.array(cols["vx"]),
                                 np.array(cols["vy"]), np.array(cols["vz"]), np.array(cols["w"]),
                                 np.array(cols["id"], np.uint64), np.array(cols["leaf"], np.int64))
    return stats
