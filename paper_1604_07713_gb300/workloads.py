"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module generates inputs only -- trees, particle populations and configuration
dictionaries shaped like the workloads of Kolobov & Arslanbekov (arXiv:1604.07713): the
capacitively coupled discharge of §3.3, the high-pressure streamer breakdown of §4 (in 2D)
and a cold-plasma oscillation.  It holds none of the method's arithmetic: no deposit,
field, push, collision or sorting step lives here.  Random numbers come from numpy's
PCG64 generator keyed by the given seed.

Configuration dictionaries use the field names of ``pic_config`` in ``include/gbpic.h``.
"""
from __future__ import annotations

import math

import numpy as np

QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
EPS0 = 8.8541878128e-12
KB_EV = 1.0  # temperatures are given in eV

BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN = 0, 1, 2
FP32, FP64 = 0, 1

DEFAULT_SEED = 160407713


def base_config(**kw) -> dict:
    cfg = dict(
        precision=FP32, n_species=2, seed=DEFAULT_SEED, dt=1e-3, eps0=1.0,
        q=[-1.0, 1.0], m=[1.0, 1836.0], qe=QE, mcc=0, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC,
        max_level=0, gas_density=0.0, gas_temperature_ev=0.026, neutral_mass=1.0,
        sigma_el=0.0, sigma_iz0=0.0, eps_th_ev=0.0, phi_left_dc=0.0, phi_left_amp=0.0,
        phi_left_freq=0.0, phi_right=0.0, rho_background=0.0, ppc_target=32, ppc_min=8,
        ppc_max=128, adapt_every=0, e_ref=1.0, refine_field=1.5, coarsen_field=1.2,
        refine_count=128, coarsen_count=32, mg_rel_tol=1e-10, mg_max_cycles=40,
        particle_capacity=0, instance=0, shape=0, implicit=0,
    )
    cfg.update(kw)
    return cfg


# ---------------------------------------------------------------------------------------
# Trees: leaves as (root, level, morton) triples of a forest of nx0 x ny0 roots
# ---------------------------------------------------------------------------------------
def _interleave(cx: np.ndarray, cy: np.ndarray) -> np.ndarray:
    cx = cx.astype(np.uint64); cy = cy.astype(np.uint64)
    out = np.zeros_like(cx)
    for b in range(16):
        out |= ((cx >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        out |= ((cy >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return out.astype(np.uint32)


def leaves_to_arrays(leaves, nx0: int):
    """{(level, gx, gy)} (global coordinates at the leaf's level) -> root, level, morton."""
    arr = np.array(sorted(leaves), dtype=np.int64).reshape(-1, 3)
    lv, gx, gy = arr[:, 0], arr[:, 1], arr[:, 2]
    root = (gx >> lv) + (gy >> lv) * nx0
    mask = (1 << lv) - 1
    mort = _interleave(gx & mask, gy & mask)
    return root.astype(np.int32), lv.astype(np.int32), mort


def _covering(leaves, lv, gx, gy):
    for l2 in range(lv, -1, -1):
        k = (l2, gx >> (lv - l2), gy >> (lv - l2))
        if k in leaves:
            return k
    return None


def balance(leaves: set, nx0: int, ny0: int, px: bool, py: bool) -> set:
    """Refine until every pair of leaves sharing a face or a corner differs by <= 1 level."""
    changed = True
    while changed:
        changed = False
        for (lv, gx, gy) in sorted(leaves, key=lambda k: -k[0]):
            if (lv, gx, gy) not in leaves or lv < 2:
                continue
            nxl, nyl = nx0 << lv, ny0 << lv
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    if dx == 0 and dy == 0:
                        continue
                    x, y = gx + dx, gy + dy
                    if not (0 <= x < nxl):
                        if not px:
                            continue
                        x %= nxl
                    if not (0 <= y < nyl):
                        if not py:
                            continue
                        y %= nyl
                    c = _covering(leaves, lv, x, y)
                    if c is not None and c[0] < lv - 1:
                        leaves.discard(c)
                        l2, a, b = c
                        for k in range(4):
                            leaves.add((l2 + 1, 2 * a + (k & 1), 2 * b + (k >> 1)))
                        changed = True
    return leaves


def random_tree(nx0: int, ny0: int, lmax: int, p_refine: float, seed: int,
                px: bool = False, py: bool = False):
    """Random 2:1-balanced forest: each leaf below lmax is refined with probability p."""
    rng = np.random.default_rng(seed)
    leaves = {(0, i, j) for i in range(nx0) for j in range(ny0)}
    for lv in range(lmax):
        for k in sorted(leaves):
            if k[0] == lv and rng.random() < p_refine:
                leaves.discard(k)
                for c in range(4):
                    leaves.add((lv + 1, 2 * k[1] + (c & 1), 2 * k[2] + (c >> 1)))
    leaves = balance(leaves, nx0, ny0, px, py)
    return leaves_to_arrays(leaves, nx0)


def region_tree(nx0: int, ny0: int, lmax: int, refine_fn, px=False, py=False):
    """Tree refined wherever ``refine_fn(level, xc, yc, h)`` (unit = root side) is True."""
    leaves = {(0, i, j) for i in range(nx0) for j in range(ny0)}
    for lv in range(lmax):
        h = 1.0 / (1 << lv)
        for k in sorted(leaves):
            if k[0] != lv:
                continue
            xc, yc = (k[1] + 0.5) * h, (k[2] + 0.5) * h
            if refine_fn(lv, xc, yc, h):
                leaves.discard(k)
                for c in range(4):
                    leaves.add((lv + 1, 2 * k[1] + (c & 1), 2 * k[2] + (c >> 1)))
    leaves = balance(leaves, nx0, ny0, px, py)
    return leaves_to_arrays(leaves, nx0)


# ---------------------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------------------
def cold_plasma(n_side=64, ppc=16, amp=0.01, dt=0.05, seed=DEFAULT_SEED, precision=FP64,
                quiet=False):
    """Periodic unit box, n_side^2 level-0 cells, ppc electrons per cell, uniform random
    positions (or, with ``quiet``, a regular sub-lattice of sqrt(ppc)^2 points per cell)
    displaced by a 1% cosine density mode in x, zero velocity; immobile uniform ion
    background; normalised units eps0 = m_e = n0 = 1, q_e = -1 (omega_p = 1)."""
    rng = np.random.default_rng(seed)
    n = n_side * n_side * ppc
    if quiet:
        k = int(round(math.sqrt(ppc)))
        g = (np.arange(n_side * k) + 0.5) / (n_side * k)
        X, Y = np.meshgrid(g, g, indexing="xy")
        x0, y = X.reshape(-1), Y.reshape(-1)
    else:
        x0 = rng.random(n); y = rng.random(n)
    x = x0 - amp / (2 * np.pi) * np.sin(2 * np.pi * x0)
    x = np.mod(x, 1.0)
    x[x >= 1.0] = 0.0
    cfg = base_config(precision=precision, n_species=1, dt=dt, eps0=1.0, q=[-1.0], m=[1.0],
                      qe=1.0, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC, rho_background=1.0,
                      mg_rel_tol=1e-13 if precision == FP64 else 1e-10)
    mesh = dict(nx0=n_side, ny0=n_side, h0=1.0 / n_side, lmax=0)
    z = np.zeros(n)
    parts = {0: dict(x=x, y=y, vx=z.copy(), vy=z.copy(), vz=z.copy(), w=np.full(n, 1.0 / n))}
    return cfg, mesh, parts


def ccp(nx=512, ny=16, ppc=100, lx=0.067, seed=DEFAULT_SEED, precision=FP32, volt=200.0,
        freq=13.56e6, n0=1e15, ng=9.6e20, te=2.5, ti=0.026, mi_amu=4.0):
    """Capacitively coupled discharge: plates at x = 0 (RF) and x = Lx (ground), periodic in
    y, square cells of side Lx/nx; electrons and ions Maxwellian at te / ti (eV), uniform
    positions, ppc macro-particles per cell and species; analytic cross sections."""
    rng = np.random.default_rng(seed)
    h = lx / nx
    mi = mi_amu * AMU
    n = nx * ny * ppc
    w = n0 * h * h / ppc
    parts = {}
    for s, (m, T) in enumerate(((ME, te), (mi, ti))):
        x = rng.random(n) * (nx * h); y = rng.random(n) * (ny * h)
        vt = math.sqrt(T * QE / m)
        v = rng.standard_normal((3, n)) * vt
        parts[s] = dict(x=x, y=y, vx=v[0], vy=v[1], vz=v[2], w=np.full(n, w))
    cfg = base_config(precision=precision, n_species=2, dt=1.0 / (400.0 * freq), eps0=EPS0,
                      q=[-QE, QE], m=[ME, mi], qe=QE, mcc=1, bc_x=BC_DIRICHLET,
                      bc_y=BC_PERIODIC, gas_density=ng, gas_temperature_ev=ti,
                      neutral_mass=mi, sigma_el=6e-20, sigma_iz0=1e-20, eps_th_ev=24.6,
                      phi_left_amp=volt, phi_left_freq=freq, phi_right=0.0,
                      mg_rel_tol=1e-10 if precision == FP32 else 1e-13)
    mesh = dict(nx0=nx, ny0=ny, h0=h, lmax=0)
    return cfg, mesh, parts


def streamer_tree(nx0=128, lmax=4, radius=0.18, length=0.55, box=1.0):
    """Quadtree of the 2D streamer: refined to lmax inside a channel along x through the
    box centre, coarser outside (2:1 balanced)."""
    def refine(lv, xc, yc, h):
        X, Y = xc / nx0, yc / nx0  # unit box coordinates
        r = radius * (0.5 ** max(0, lv - 1))
        inside = abs(Y - 0.5) < r + h / nx0 and (0.5 - length / 2 - h / nx0) < X < (0.5 + length / 2 + h / nx0)
        return inside
    return region_tree(nx0, nx0, lmax, refine)


def streamer(n_particles=200_000, nx0=128, lmax=4, seed=DEFAULT_SEED, precision=FP32,
             box=0.01, e0=3e6, ng=3.2e24, dt=1e-13, sigma=2e-4, tree=None):
    """2D streamer in a 1 cm box: uniform background field E0 along -x (phi = 0 at x = 0,
    E0*Lx at x = Lx), Neumann in y, absorbing walls; a neutral Gaussian seed of electrons
    and ions (sigma = 0.2 mm) at the centre elongated along x; ionization MCC with the
    analytic cross sections; split/merge toward 32 per leaf in the 8-128 band."""
    rng = np.random.default_rng(seed)
    h0 = box / nx0
    if tree is None:
        tree = streamer_tree(nx0, lmax)
    n = n_particles // 2
    parts = {}
    mi = 4.0 * AMU
    for s, (m, T) in enumerate(((ME, 5.0), (mi, 0.026))):
        x = 0.5 * box + rng.standard_normal(n) * sigma * 4.0
        y = 0.5 * box + rng.standard_normal(n) * sigma
        x = np.clip(x, 1e-6 * box, box * (1 - 1e-6)); y = np.clip(y, 1e-6 * box, box * (1 - 1e-6))
        vt = math.sqrt(T * QE / m)
        v = rng.standard_normal((3, n)) * vt
        parts[s] = dict(x=x, y=y, vx=v[0], vy=v[1], vz=v[2], w=np.full(n, 1e13 / n))
    cfg = base_config(precision=precision, n_species=2, dt=dt, eps0=EPS0, q=[-QE, QE],
                      m=[ME, mi], qe=QE, mcc=1, bc_x=BC_DIRICHLET, bc_y=BC_NEUMANN,
                      max_level=lmax, gas_density=ng, gas_temperature_ev=0.026, neutral_mass=mi,
                      sigma_el=6e-20, sigma_iz0=1e-20, eps_th_ev=24.6, phi_left_dc=0.0,
                      phi_right=e0 * box, e_ref=e0, adapt_every=10)
    root, level, mort = tree
    mesh = dict(nx0=nx0, ny0=nx0, h0=h0, lmax=lmax, root=root, level=level, morton=mort)
    return cfg, mesh, parts


def streamer_snapshot(n_particles=50_000_000, nx0=128, lmax=4, seed=DEFAULT_SEED, precision=FP32,
                      box=0.01, e0=3e6, ng=3.2e24, dt=1e-13, n_e=1e19):
    """A grown 2D streamer: electrons and ions (half each) in a channel along x through the
    box centre (uniform over the middle half of the box in x with Gaussian ends, Gaussian
    across with sigma = 0.5 mm), electrons Maxwellian at 5 eV and ions at 0.026 eV; weights
    give a channel density of about n_e.  Same physics and walls as ``streamer``; the mesh
    starts as the uniform root grid and is refined on the device by adaptation."""
    rng = np.random.default_rng(seed)
    n = n_particles // 2
    h0 = box / nx0
    sig_y = 0.05 * box
    parts = {}
    mi = 4.0 * AMU
    area = 0.5 * box * (2.5 * sig_y)
    w = n_e * area / n
    for s, (m, T) in enumerate(((ME, 5.0), (mi, 0.026))):
        u = rng.random(n)
        x = 0.25 * box + 0.5 * box * u
        tail = rng.random(n) < 0.1
        x[tail] = 0.5 * box + 0.3 * box * rng.standard_normal(int(tail.sum()))
        y = 0.5 * box + sig_y * rng.standard_normal(n)
        x = np.clip(x, 1e-4 * box, box * (1 - 1e-4)); y = np.clip(y, 1e-4 * box, box * (1 - 1e-4))
        vt = math.sqrt(T * QE / m)
        v = rng.standard_normal((3, n)) * vt
        parts[s] = dict(x=x, y=y, vx=v[0], vy=v[1], vz=v[2], w=np.full(n, w))
    cfg = base_config(precision=precision, n_species=2, dt=dt, eps0=EPS0, q=[-QE, QE],
                      m=[ME, mi], qe=QE, mcc=1, bc_x=BC_DIRICHLET, bc_y=BC_NEUMANN,
                      max_level=lmax, gas_density=ng, gas_temperature_ev=0.026, neutral_mass=mi,
                      sigma_el=6e-20, sigma_iz0=1e-20, eps_th_ev=24.6, phi_left_dc=0.0,
                      phi_right=e0 * box, e_ref=e0, adapt_every=10, mg_rel_tol=1e-8)
    mesh = dict(nx0=nx0, ny0=nx0, h0=h0, lmax=lmax)
    return cfg, mesh, parts


def ensemble(n_instances=256, seed=DEFAULT_SEED, precision=FP32, lx_per_cell=0.067 / 512):
    """Batched capacitively coupled discharges of uneven size: per instance x-cells drawn
    from {64, 80, ..., 512} (multiples of 16 so that the root grid coarsens), 16 y-cells,
    20-200 macro-particles per cell and species, RF amplitude 100-400 V, gas density
    log-uniform in 3e20-3e21 m^-3, otherwise the CCP physics; each instance has its own
    seed and Philox instance word.  Returns a list of (cfg, mesh, parts_factory) where
    parts_factory() draws that instance's particles (so the host holds one at a time)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        nx = int(rng.integers(4, 33)) * 16
        ppc = int(rng.integers(20, 201))
        volt = float(rng.uniform(100.0, 400.0))
        ng = float(np.exp(rng.uniform(np.log(3e20), np.log(3e21))))
        s_i = int(rng.integers(0, 2**31))
        def factory(nx=nx, ppc=ppc, volt=volt, ng=ng, s_i=s_i):
            return ccp(nx=nx, ny=16, ppc=ppc, lx=lx_per_cell * nx, seed=s_i, precision=precision,
                       volt=volt, ng=ng)[2]
        cfg, mesh, _ = ccp(nx=nx, ny=16, ppc=1, lx=lx_per_cell * nx, seed=s_i, precision=precision,
                           volt=volt, ng=ng)
        cfg["instance"] = i % 256
        cfg["mg_rel_tol"] = 1e-8
        out.append((cfg, mesh, factory, nx * 16 * ppc * 2))
    return out
