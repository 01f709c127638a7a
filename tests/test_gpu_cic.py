"""Cloud-in-cell shapes on uniform meshes (§3: CIC-EM, momentum conserving; CIC-EC, energy
conserving) on the GPU against the FP64 oracle from identical state: deposit, solve and field
within 1e-12 (FP64) or 1e-5 (FP32; rho 1e-6); one step with ionization bit-exact in list
order (FP64); several cold-plasma steps tracking the oracle; and CIC-EM's momentum
conservation on a periodic box."""
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
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _pair(cfg, mesh, parts):
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], 0, cfg["bc_x"], cfg["bc_y"])
    sim = O.Sim(cfg, M)
    ctx = G.Context(cfg)
    ctx.set_mesh_dict(mesh)
    for s in sorted(parts):
        sim.load(s, **parts[s])
        ctx.load(s, **parts[s])
    return sim, ctx


@pytest.mark.parametrize("shape", [G.PIC_SHAPE_CIC_EM, G.PIC_SHAPE_CIC_EC])
@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_cic_fields_and_one_step_match_the_oracle(shape, precision):
    cfg, mesh, parts = W.ccp(nx=32, ny=8, ppc=40, seed=5, precision=precision, te=30.0, ng=3e21)
    cfg.update(shape=shape, mg_rel_tol=1e-13 if precision == W.FP64 else 1e-11)
    cfg["dt"] *= 4
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        rho_o, phi_o, _ = sim.fields()
        ctx.compute_fields()
        rho, phi = ctx.fields(G.PIC_FIELD_RHO), ctx.fields(G.PIC_FIELD_PHI)
        tol = 1e-12 if precision == W.FP64 else 1e-5
        assert _rel(rho, rho_o) < (1e-13 if precision == W.FP64 else 1e-6)
        assert _rel(phi, phi_o) < tol
        sim.step(1)
        ctx.step(1)
        g = [ctx.particles(s) for s in (0, 1)]
    assert sim.species[1].n > parts[1]["x"].size + 20, "the case must exercise ionization"
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


@pytest.mark.parametrize("shape", [G.PIC_SHAPE_CIC_EM, G.PIC_SHAPE_CIC_EC])
def test_cic_cold_plasma_tracks_the_oracle_fp64(shape):
    cfg, mesh, parts = W.cold_plasma(n_side=32, ppc=4, dt=0.05)
    cfg["shape"] = shape
    sim, ctx = _pair(cfg, mesh, parts)
    with ctx:
        sim.step(10)
        ctx.step(10)
        g = ctx.particles(0)
    sp = sim.species[0]
    assert np.array_equal(g["id"], sp.id)
    assert np.abs(g["x"] - sp.x).max() < 1e-10
    assert np.abs(g["vx"] - sp.vx).max() < 1e-10 * max(1e-30, np.abs(sp.vx).max()) + 1e-14


def test_cic_em_conserves_momentum_on_the_gpu():
    """CIC-EM gathers with the deposit's weights: in a periodic box without collisions the
    total momentum of the electrons over a step changes only by rounding (NGP's corner gather
    and CIC-EC do not conserve it)."""
    def momentum_change(shape):
        cfg, mesh, parts = W.cold_plasma(n_side=32, ppc=4, dt=0.05, amp=0.3)
        cfg["shape"] = shape
        with G.Context(cfg) as ctx:
            ctx.set_mesh_dict(mesh)
            ctx.load(0, **parts[0])
            p0 = ctx.particles(0)
            ctx.step(1)
            p1 = ctx.particles(0)
        o0, o1 = np.argsort(p0["id"]), np.argsort(p1["id"])
        dP = np.array([np.sum(p1["w"][o1] * p1[k][o1]) - np.sum(p0["w"][o0] * p0[k][o0]) for k in ("vx", "vy")])
        scale = np.sum(p1["w"] * np.hypot(p1["vx"], p1["vy"]))
        return np.abs(dP).max() / scale
    assert momentum_change(G.PIC_SHAPE_CIC_EM) < 1e-12
    assert momentum_change(G.PIC_SHAPE_NGP) > 1e-9
