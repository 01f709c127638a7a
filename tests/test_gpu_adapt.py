"""GPU mesh adaptation and split/merge (§3.1, §4.3) against the oracle, from identical state.

FP64 mode: the new tree, every particle's leaf and the cell-list order (ids) are bit-exact,
positions and velocities within 1e-12.  FP32 mode: inputs are chosen exactly representable
(dyadic box, float32 positions and velocities) so that every integer decision (refinement
flags, child by position, energy bin) is taken on identical values; then the tree and the
list order are bit-exact and the merged / split values agree within FP32 rounding.
"""
import numpy as np
import pytest

import oracle as O
import paper_1604_07713_gb300 as G
from paper_1604_07713_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    G.build()
    O.build()


def _pair(cfg, mesh, parts):
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], mesh.get("lmax", 0), cfg["bc_x"], cfg["bc_y"],
               mesh.get("root"), mesh.get("level"), mesh.get("morton"))
    sim = O.Sim(cfg, M)
    for s in sorted(parts):
        sim.load(s, **parts[s])
    ctx = G.Context(cfg)
    ctx.set_mesh_dict(mesh)
    for s in sorted(parts):
        ctx.load(s, **parts[s])
    return sim, ctx


def _compare(sim, ctx, tol_rel, exact_order=True):
    r, m, lv = ctx.mesh()
    M = sim.mesh
    assert np.array_equal(r, M.root) and np.array_equal(m, M.morton) and np.array_equal(lv, M.level)
    for s, sp in enumerate(sim.species):
        g = ctx.particles(s)
        assert g["x"].size == sp.n
        if exact_order:
            assert np.array_equal(g["id"], sp.id), f"species {s}: list order"
            assert np.array_equal(g["leaf"].astype(np.int64), sp.leaf)
        o = np.argsort(g["id"]); oo = np.argsort(sp.id)
        for k, ref in (("x", sp.x), ("y", sp.y), ("vx", sp.vx), ("vy", sp.vy), ("w", sp.w)):
            a, b = g[k][o], ref[oo]
            assert np.abs(a - b).max() <= tol_rel * max(1e-300, np.abs(b).max()), (s, k)


def test_adapt_and_split_merge_fp64_bit_exact_structure():
    tree = W.streamer_tree(nx0=16, lmax=3)
    cfg, mesh, parts = W.streamer(n_particles=40000, nx0=16, lmax=3, precision=W.FP64, tree=tree)
    cfg["mg_rel_tol"] = 1e-13
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        sim.fields(); ctx.compute_fields()
        st = sim.adapt()
        ctx.adapt()
        assert st["mesh"]["coarsened"] > 0 and st["particles"]["merged"] > 0 and st["particles"]["split"] > 0
        _compare(sim, ctx, 1e-12)
        # and the cycle continues on the adapted mesh
        sim.step(2)
        ctx.step(2)
        _compare(sim, ctx, 1e-11)


def _dyadic_case(precision, seed=3):
    """Unit box, 8 x 8 roots, up to 3 levels; a dense blob (merging, refinement by count),
    a sparse halo (splitting) and empty corners (coarsening); float32-exact inputs."""
    rng = np.random.default_rng(seed)
    r, l, m = W.region_tree(8, 8, 2, lambda lv, xc, yc, h: abs(xc / 8 - 0.5) < 0.3 and abs(yc / 8 - 0.5) < 0.3)
    mesh = dict(nx0=8, ny0=8, h0=0.125, lmax=3, root=r, level=l, morton=m)
    n1, n2 = 6000, 300
    x = np.concatenate([0.5 + 0.03 * rng.standard_normal(n1), 0.2 + 0.6 * rng.random(n2)])
    y = np.concatenate([0.5 + 0.03 * rng.standard_normal(n1), 0.2 + 0.6 * rng.random(n2)])
    x = np.clip(x, 0.01, 0.99).astype(np.float32).astype(np.float64)
    y = np.clip(y, 0.01, 0.99).astype(np.float32).astype(np.float64)
    v = rng.standard_normal((3, x.size)).astype(np.float32).astype(np.float64)
    w = np.full(x.size, 0.25)
    cfg = W.base_config(precision=precision, n_species=1, q=[-1.0], m=[1.0], qe=1.0, eps0=1.0,
                        bc_x=W.BC_DIRICHLET, bc_y=W.BC_NEUMANN, max_level=3, refine_count=128,
                        coarsen_count=32, e_ref=1e30, ppc_min=8, ppc_max=128, ppc_target=32,
                        mg_rel_tol=1e-12)
    parts = {0: dict(x=x, y=y, vx=v[0], vy=v[1], vz=v[2], w=w)}
    return cfg, mesh, parts


@pytest.mark.parametrize("precision", [W.FP32, W.FP64])
def test_adapt_split_merge_dyadic_exact_decisions(precision):
    cfg, mesh, parts = _dyadic_case(precision)
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        sim.fields(); ctx.compute_fields()
        st = sim.adapt()
        ctx.adapt()
        assert st["mesh"]["refined"] > 0 and st["mesh"]["coarsened"] > 0
        assert st["particles"]["merged"] > 0 and st["particles"]["split"] > 0
        _compare(sim, ctx, 1e-6 if precision == W.FP32 else 1e-13)
        c = ctx.fields(G.PIC_FIELD_COUNT_E)
        assert c[c > 0].min() >= 8 and c.max() <= 128


def test_adapt_with_crowded_lists_lays_them_out_first_fp64():
    # a hard capacity equal to the population leaves almost no tail: the adaptation first
    # lays every list out again (a compaction), then refines / coarsens in place
    cfg, mesh, parts = _dyadic_case(W.FP64)
    cfg.update(ppc_min=1, ppc_max=1 << 20, particle_capacity=parts[0]["x"].size)
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        sim.fields(); ctx.compute_fields()
        st = sim.adapt()
        ctx.adapt()
        assert st["mesh"]["refined"] > 0 and st["mesh"]["coarsened"] > 0
        _compare(sim, ctx, 1e-13)
        assert G.pic_get_list_stats(ctx.ctx, 0, 0)[0] >= 1  # the compaction ran
        sim.step(2)
        ctx.step(2)
        _compare(sim, ctx, 1e-11)


def test_adapt_fp32_with_the_field_criterion_on():
    """FP32 state with the |E| criterion active: the threshold is put in a gap of the oracle's
    centre |E| values (every |E| at least 1e-6 away from the refine and coarsen thresholds;
    |E| comes from the FP64 potential on both sides), so the refinement decisions, the tree
    and the list order are bit-exact; more leaves refine than the count criterion alone asks."""
    cfg, mesh, parts = _dyadic_case(W.FP32)
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], mesh["lmax"], cfg["bc_x"], cfg["bc_y"], mesh["root"],
               mesh["level"], mesh["morton"])
    probe = O.Sim(cfg, M)
    probe.load(0, **parts[0])
    probe.fields()
    em = np.sort(M.cell_emag(probe.phi, probe.last_walls))
    ok = lambda t: np.all(np.abs(em - t) > 1e-6 * t) and np.all(np.abs(em - 0.8 * t) > 1e-6 * t)
    lo = int(0.7 * em.size)
    gaps = [(em[i + 1] - em[i], i) for i in range(lo, em.size - 1)]
    thr = None
    for _, i in sorted(gaps, reverse=True):
        t = 0.5 * (em[i] + em[i + 1])
        if ok(t):
            thr = t
            break
    assert thr is not None
    cfg["e_ref"] = thr / cfg["refine_field"]            # refine above thr, coarsen below 0.8 thr
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        sim.fields(); ctx.compute_fields()
        cnt = sim.counts(0)
        by_count = int(np.count_nonzero((cnt > cfg["refine_count"]) & (sim.mesh.level < mesh["lmax"])))
        st = sim.adapt()
        ctx.adapt()
        assert st["mesh"]["refined"] > by_count + 5
        _compare(sim, ctx, 1e-6)
