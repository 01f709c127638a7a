"""The direct implicit scheme (§3 DIPIC) on the GPU against the FP64 oracle from identical
state: the susceptibility operator's fields (uniform, AMR and multi-block meshes, a periodic
cold plasma), one implicit step with ionization bit-exact in list order (FP64) or within the
FP32 bars, several cold-plasma steps tracking the oracle at omega_p dt = 0.5, and the
scheme's stability at omega_p dt = 2.5 where the leapfrog grows."""
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


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, float) - b) / (nb if nb > 0 else 1.0)


def _pair(cfg, mesh, parts):
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], mesh.get("lmax", 0), cfg["bc_x"], cfg["bc_y"],
               mesh.get("root"), mesh.get("level"), mesh.get("morton"))
    sim = O.Sim(cfg, M)
    ctx = G.Context(cfg)
    ctx.set_mesh_dict(mesh)
    for s in sorted(parts):
        sim.load(s, **parts[s])
        ctx.load(s, **parts[s])
    return sim, ctx


def _amr_mesh(nx0, ny0, h0, lmax, seed, px=False, py=False):
    r, l, m = W.random_tree(nx0, ny0, lmax, 0.3, seed, px, py)
    return dict(nx0=nx0, ny0=ny0, h0=h0, lmax=lmax, root=r, level=l, morton=m)


def _dense_ccp(precision, nx=32, ny=8, ppc=40, seed=5, amr=False, boost=100.0):
    # a denser CCP (n0 x boost) with ionization at 4 dt: omega_p dt ~ 13 on the electrons at
    # the default boost, so the susceptibility is far from 1
    cfg, mesh, parts = W.ccp(nx=nx, ny=ny, ppc=ppc, seed=seed, precision=precision, te=30.0, ng=3e21)
    for s in parts:
        parts[s]["w"] = parts[s]["w"] * boost
    cfg.update(implicit=1, mg_rel_tol=1e-13 if precision == W.FP64 else 1e-11)
    cfg["dt"] *= 4
    if amr:
        mesh = _amr_mesh(nx, ny, mesh["h0"], 2, 5, py=True)
        cfg["max_level"] = 2
    return cfg, mesh, parts


@pytest.mark.parametrize("amr", [False, True])
@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_implicit_fields_and_one_step_match_the_oracle(precision, amr):
    cfg, mesh, parts = _dense_ccp(precision, amr=amr)
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        chi = sim.kappa() - 1.0
        assert chi.max() > 0.5, "the susceptibility must matter"
        rho_o, phi_o, E_o = sim.fields()
        ctx.compute_fields()
        rho, phi = ctx.fields(G.PIC_FIELD_RHO), ctx.fields(G.PIC_FIELD_PHI)
        E = ctx.fields(G.PIC_FIELD_NODE_E)
        tol = 1e-12 if precision == W.FP64 else 1e-5
        assert _rel(rho, rho_o) < (1e-13 if precision == W.FP64 else 1e-6)
        assert _rel(phi, phi_o) < tol and _rel(E.reshape(-1), E_o.reshape(-1)) < tol
        # the field differs from the explicit one of the same charge
        phi_exp = sim.mesh.solve_poisson(rho_o * sim.mesh.area() / cfg["eps0"], sim.walls())
        assert _rel(phi, phi_exp) > 1e-3
        sim.step(1)
        ctx.step(1)
        g = [ctx.particles(s) for s in (0, 1)]
        phi_o1 = sim.phi
        phi1 = ctx.fields(G.PIC_FIELD_PHI)
    assert sim.species[1].n > parts[1]["x"].size + 20, "the case must exercise ionization"
    assert _rel(phi1, phi_o1) < tol  # the step's own field: the predicted charge, the susceptibility
    for s in (0, 1):
        sp = sim.species[s]
        if precision == W.FP64:
            assert np.array_equal(g[s]["id"], sp.id), f"species {s}: cell-list order"
            assert np.array_equal(g[s]["leaf"].astype(np.int64), sp.leaf)
            for k, ref in (("x", sp.x), ("y", sp.y), ("vx", sp.vx), ("vy", sp.vy), ("vz", sp.vz)):
                assert np.abs(g[s][k] - ref).max() <= 1e-12 * np.abs(ref).max(), (s, k)
        else:
            # FP32: the particles common to both (collision decisions inside the rounding
            # margin may differ) agree in position to 1e-5 of a cell
            o = np.argsort(sp.id); a = np.argsort(g[s]["id"])
            common, ia, io = np.intersect1d(g[s]["id"][a], sp.id[o], return_indices=True)
            assert common.size >= 0.999 * sp.n
            dx = np.abs(g[s]["x"][a][ia] - sp.x[o][io])
            assert np.quantile(dx, 0.999) <= 1e-5 * mesh["h0"]


def test_implicit_fields_multiblock_levels_fp64():
    # more than 8192 leaves: the multi-block levels and the one-block tail carry kappa
    # (2 particles per cell: kappa jumps from cell to cell, which the averaged coarse
    # operators follow slowly, so the density is not boosted and the cycle bound is higher)
    cfg, mesh, parts = _dense_ccp(W.FP64, nx=96, ny=64, ppc=2, boost=1.0)
    mesh = _amr_mesh(96, 64, mesh["h0"], 1, 11, py=True)
    cfg.update(max_level=1, mg_max_cycles=200)
    assert mesh["root"].size > 8192
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        rho_o, phi_o, E_o = sim.fields()
        ctx.compute_fields()
        phi = ctx.fields(G.PIC_FIELD_PHI)
        c = ctx.counts()
    assert _rel(phi, phi_o) < 1e-12
    assert c["mg_rel_res"] <= cfg["mg_rel_tol"]
    print("multi-block implicit solve: cycles", c["mg_cycles"])


def _cold(dt, implicit=1):
    cfg, mesh, parts = W.cold_plasma(n_side=32, ppc=4, dt=dt)
    cfg["implicit"] = implicit
    return cfg, mesh, parts


def test_implicit_cold_plasma_tracks_the_oracle_fp64():
    # omega_p dt = 0.5, fully periodic (the singular, zero-mean solve with kappa)
    cfg, mesh, parts = _cold(0.5)
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        sim.step(10)
        ctx.step(10)
        g = ctx.particles(0)
    sp = sim.species[0]
    assert np.array_equal(g["id"], sp.id)
    assert np.abs(g["x"] - sp.x).max() < 1e-10
    assert np.abs(g["vx"] - sp.vx).max() < 1e-10 * max(1e-30, np.abs(sp.vx).max()) + 1e-14


def test_implicit_step_is_stable_where_leapfrog_grows():
    # omega_p dt = 2.5 on a 20 % density mode: the implicit field energy decays, the
    # leapfrog's grows (GPU alone; the oracle's pins check the same on its side)
    def field_energy(implicit, steps):
        cfg, mesh, parts = W.cold_plasma(n_side=64, ppc=16, dt=2.5, quiet=True, amp=0.2)
        cfg["implicit"] = implicit
        out = []
        with G.Context(cfg) as ctx:
            ctx.set_mesh_dict(mesh)
            ctx.load(0, **parts[0])
            for _ in range(steps):
                ctx.step(1)
                e = ctx.fields(G.PIC_FIELD_NODE_E)
                out.append(float(np.sum(e * e)))
        return np.array(out)
    imp = field_energy(1, 6)
    exp_ = field_energy(0, 6)
    # (the implicit mode decays to the NGP noise floor of the quiet start within 3 steps)
    assert imp[3:].max() < 0.1 * imp[0], imp
    assert exp_.max() > 10.0 * exp_[0], exp_


def test_implicit_needs_the_ngp_shape():
    cfg, mesh, parts = _cold(0.5)
    cfg["shape"] = G.PIC_SHAPE_CIC_EM
    with pytest.raises(G.PicError) as e:
        G.Context(cfg)
    assert e.value.status == G.PIC_EINVAL
