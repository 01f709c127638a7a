"""Failure paths and checkpoint/resume through the C ABI on the GPU.  Every failure is made on
the host (an injected allocation failure, a bounded closure given a smaller bound, a NaN in
the input data): no test faults, traps or hangs the GPU.

- The explicit-PIC limits of §3 are checked when the electrons are loaded.
- An allocation failure returns PIC_ENOMEM and leaves the context usable.
- The adaptation's balance closure returns PIC_ETIMEOUT at its bound, before the mesh
  changes, and the context carries on.
- A non-finite charge density is reported by the Poisson solve's status.
- A checkpoint restored into a fresh context continues bit for bit like the original run.
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


def _ctx(cfg, mesh, parts):
    ctx = G.Context(cfg)
    ctx.set_mesh_dict(mesh)
    for s in sorted(parts):
        ctx.load(s, **parts[s])
    return ctx


# ---------------------------------------------------------------------------------------
# §3 explicit-PIC limits
# ---------------------------------------------------------------------------------------
def test_loading_electrons_checks_the_explicit_pic_limits():
    # the discharge's cells (6.7 cm / 512): h / lambda_D = 0.35 and omega_pe dt = 0.33 on average
    cfg, mesh, parts = W.ccp(nx=64, ny=8, ppc=50, seed=3, precision=W.FP32, lx=0.067 / 8)
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        assert ctx.load(0, **parts[0]) == G.PIC_OK, G.pic_last_error()
        st, dx_ld, wdt, te = ctx.stability()
    # independent evaluation from the loaded arrays (as the FP32 state holds them): per-cell
    # weight sums on the uniform mesh
    p = {k: (v.astype(np.float32).astype(np.float64) if k in ("vx", "vy", "vz", "w") else v)
         for k, v in parts[0].items()}
    h = mesh["h0"]
    ix = np.floor(p["x"] / h).astype(int); iy = np.floor(p["y"] / h).astype(int)
    Wc = np.zeros((mesh["ny0"], mesh["nx0"]))
    np.add.at(Wc, (iy, ix), p["w"])
    w = p["w"]
    v = np.stack([p["vx"], p["vy"], p["vz"]])
    var = ((w * v * v).sum(1) / w.sum() - ((w * v).sum(1) / w.sum()) ** 2).sum()
    te_ref = W.ME * var / 3 / W.QE
    st_ref, a_ref, b_ref = G.pic_stability_limits(cfg, Wc.max() / h ** 2, Wc.max(), te_ref)
    assert st == st_ref == G.PIC_OK
    assert abs(te / te_ref - 1) < 1e-9 and abs(dx_ld / a_ref - 1) < 1e-9 and abs(wdt / b_ref - 1) < 1e-9, \
        (te / te_ref - 1, dx_ld / a_ref - 1, wdt / b_ref - 1)
    assert abs(te / 2.5 - 1) < 0.02                      # the 2.5 eV Maxwellian
    # 100 times the density: omega_pe dt = 3.3 > 1, the load warns and still loads
    dense = dict(parts[0], w=parts[0]["w"] * 100.0)
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        assert ctx.load(0, **dense) == G.PIC_WARN_STABILITY
        assert "omega_pe dt" in G.pic_last_error()
        assert ctx.counts()["n_e"] == p["x"].size
        st, dx_ld, wdt, _ = ctx.stability()
        assert st == G.PIC_WARN_STABILITY and abs(wdt / (10 * b_ref) - 1) < 1e-6


# ---------------------------------------------------------------------------------------
# injected faults
# ---------------------------------------------------------------------------------------
def test_injected_allocation_failure_returns_enomem_and_the_context_recovers():
    cfg, mesh, parts = W.ccp(nx=32, ny=8, ppc=20, seed=4, precision=W.FP32)
    with G.Context(cfg) as ctx:
        G.pic_inject_fault(ctx.ctx, G.PIC_FAULT_ALLOC, 3)
        with pytest.raises(G.PicError) as e:
            ctx.set_mesh_dict(mesh)
        assert e.value.status == G.PIC_ENOMEM and "injected" in str(e.value)
        # the fault fires once; the same calls then succeed and the run matches a clean one
        ctx.set_mesh_dict(mesh)
        for s in (0, 1):
            ctx.load(s, **parts[s])
        G.pic_inject_fault(ctx.ctx, G.PIC_FAULT_ALLOC, 0)
        with pytest.raises(G.PicError) as e:
            ctx.particles(0)                             # its read-back buffers are allocated
        assert e.value.status == G.PIC_ENOMEM
        ctx.step(3)
        a = [ctx.particles(s) for s in (0, 1)]
    with _ctx(cfg, mesh, parts) as ref:
        ref.step(3)
        b = [ref.particles(s) for s in (0, 1)]
    for s in (0, 1):
        for k in a[s]:
            assert np.array_equal(a[s][k], b[s][k]), (s, k)


def _deep_refinement_case():
    # a level-2 region next to level-0 leaves; 30 electrons in one level-2 leaf make it refine,
    # which forces a chain of neighbours to refine (the closure needs more than one sweep)
    r, l, m = W.region_tree(4, 4, 2, lambda lv, xc, yc, h: abs(xc / 4 - 0.4) < 0.2 and abs(yc / 4 - 0.4) < 0.2)
    cfg = W.base_config(precision=W.FP64, n_species=1, q=[-1.0], m=[1.0], bc_x=W.BC_DIRICHLET,
                        bc_y=W.BC_NEUMANN, max_level=3, refine_count=20, coarsen_count=-1, e_ref=1e30)
    mesh = dict(nx0=4, ny0=4, h0=0.25, lmax=3, root=r, level=l, morton=m)
    M = O.Mesh(4, 4, 0.25, 3, O.BC_DIRICHLET, O.BC_NEUMANN, r, l, m)
    deep = np.nonzero(M.level == M.level.max())[0][0]
    h = M.s[deep] * M.hf
    rng = np.random.default_rng(1)
    x = M.ix[deep] * M.hf + h * (0.05 + 0.9 * rng.random(30))
    y = M.iy[deep] * M.hf + h * (0.05 + 0.9 * rng.random(30))
    z = np.zeros(30)
    parts = {0: dict(x=x, y=y, vx=z, vy=z, vz=z, w=np.full(30, 1e-9))}
    return cfg, mesh, parts, M


def test_balance_closure_bound_returns_etimeout_before_the_mesh_changes():
    cfg, mesh, parts, M = _deep_refinement_case()
    sim = O.Sim(cfg, M)
    sim.load(0, **parts[0])
    sim.fields()
    sim.adapt(particles=False)
    with _ctx(cfg, mesh, parts) as ctx:
        ctx.compute_fields()
        before = ctx.mesh()
        G.pic_inject_fault(ctx.ctx, G.PIC_FAULT_BALANCE, 1)
        with pytest.raises(G.PicError) as e:
            ctx.adapt(G.PIC_ADAPT_MESH)
        assert e.value.status == G.PIC_ETIMEOUT
        after = ctx.mesh()
        assert all(np.array_equal(a, b) for a, b in zip(before, after))
        G.pic_inject_fault(ctx.ctx, G.PIC_FAULT_NONE)
        ctx.adapt(G.PIC_ADAPT_MESH)
        r, m, lv = ctx.mesh()
        g = ctx.particles(0)
    M2 = sim.mesh
    assert np.array_equal(r, M2.root) and np.array_equal(m, M2.morton) and np.array_equal(lv, M2.level)
    assert np.array_equal(g["id"], sim.species[0].id)


def test_non_finite_charge_density_is_reported_by_the_solve():
    cfg, mesh, parts = W.ccp(nx=32, ny=8, ppc=20, seed=6, precision=W.FP32)
    bad = {s: dict(p) for s, p in parts.items()}
    bad[0]["w"] = bad[0]["w"].copy()
    bad[0]["w"][123] = np.nan
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        for s in (0, 1):
            ctx.load(s, **bad[s])
        with pytest.raises(G.PicError) as e:
            ctx.compute_fields()
        assert e.value.status == G.PIC_ENOTCONV and "non-finite" in str(e.value)
        # not poisoned: a clean population solves
        for s in (0, 1):
            ctx.load(s, **parts[s])
        ctx.compute_fields()
        assert np.isfinite(ctx.fields(G.PIC_FIELD_PHI)).all()


# ---------------------------------------------------------------------------------------
# checkpoint / resume
# ---------------------------------------------------------------------------------------
def _state(ctx, nsp):
    out = [ctx.particles(s) for s in range(nsp)]
    ctx.compute_fields(allow_notconv=True)
    return out, ctx.fields(G.PIC_FIELD_PHI), ctx.mesh(), G.pic_get_step(ctx.ctx)


def _same(a, b):
    pa, phia, ma, sa = a
    pb, phib, mb, sb = b
    assert sa == sb
    assert all(np.array_equal(x, y) for x, y in zip(ma, mb))
    assert np.array_equal(phia, phib)
    for s in range(len(pa)):
        for k in pa[s]:
            assert np.array_equal(pa[s][k], pb[s][k]), (s, k)


@pytest.mark.parametrize("precision", [W.FP32, W.FP64])
def test_checkpoint_resume_continues_bit_for_bit_ccp(precision):
    cfg, mesh, parts = W.ccp(nx=64, ny=8, ppc=30, seed=8, precision=precision, te=30.0, ng=3e21)
    with _ctx(cfg, mesh, parts) as a:
        a.step(3)
        image = a.checkpoint()
        a.step(4)
        ref = _state(a, 2)
        assert ref[0][1]["x"].size > parts[1]["x"].size   # ionization happened
    with G.Context(cfg) as b:
        b.restore(image)
        b.step(4)
        _same(_state(b, 2), ref)


def test_checkpoint_resume_continues_bit_for_bit_with_adaptation():
    tree = W.streamer_tree(nx0=16, lmax=2)
    cfg, mesh, parts = W.streamer(n_particles=20000, nx0=16, lmax=2, precision=W.FP32, tree=tree)
    cfg["mg_rel_tol"] = 1e-10

    def cycle(ctx, k):
        for i in range(k):
            ctx.step(1)
            if i % 3 == 2:
                ctx.adapt()

    with _ctx(cfg, mesh, parts) as a:
        cycle(a, 4)
        image = a.checkpoint()
        cycle(a, 5)
        ref = _state(a, 2)
    with G.Context(cfg) as b:
        b.restore(image)
        cycle(b, 5)
        _same(_state(b, 2), ref)
    # a context of another precision refuses the image, and so does a truncated one
    cfg64 = dict(cfg, precision=W.FP64)
    with G.Context(cfg64) as c:
        with pytest.raises(G.PicError) as e:
            c.restore(image)
        assert e.value.status == G.PIC_EINVAL
        with pytest.raises(G.PicError):
            c.restore(image[:100])
