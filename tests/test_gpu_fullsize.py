"""The streamer at its full size (5e7 particles, ~3.8e5 leaves after adaptation), in the launch
configuration the benchmark times: properties that hold at any size (every particle inside
the leaf that lists it, per-leaf counts, unique ids, charge conservation of the deposit), and
one step of a random sample of particles recomputed by the oracle's push and collisions from
the GPU's own corner field (FP32 against FP64: positions, velocities, leaves and absorption
within rounding; collision decisions may differ only inside the rounding margin)."""
import ctypes as C

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


def test_streamer_full_size_properties_and_sampled_step():
    cfg, mesh, parts = W.streamer_snapshot(n_particles=50_000_000, precision=W.FP32)
    rng = np.random.default_rng(20240601)
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        for s in sorted(parts):
            ctx.load(s, **parts[s])
        del parts
        # the benchmark's setup: refine the roots onto the particles, manage them, two steps
        for _ in range(mesh["lmax"] + 1):
            ctx.compute_fields(allow_notconv=True)
            ctx.adapt(G.PIC_ADAPT_MESH)
        ctx.compute_fields(allow_notconv=True)
        ctx.adapt()
        ctx.step(2)
        r, m, lv = ctx.mesh()
        M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], mesh["lmax"], cfg["bc_x"], cfg["bc_y"], r, lv, m,
                   check=False)
        assert np.array_equal(M.root, r) and np.array_equal(M.morton, m)  # the same leaf order
        assert M.nleaf > 200_000
        ctx.compute_fields()
        E = np.ascontiguousarray(ctx.fields(G.PIC_FIELD_NODE_E).reshape(-1))
        rho = ctx.fields(G.PIC_FIELD_RHO)
        counts = [ctx.fields(G.PIC_FIELD_COUNT_E), ctx.fields(G.PIC_FIELD_COUNT_I)]
        step = G.pic_get_step(ctx.ctx)
        charge, scale, sample = 0.0, 0.0, {}
        hf = M.hf
        for s in (0, 1):
            p = ctx.particles(s)
            leaf = p["leaf"].astype(np.int64)
            x0, y0, side = M.ix[leaf] * hf, M.iy[leaf] * hf, M.s[leaf] * hf
            tol = 1e-12 * mesh["h0"]
            assert np.all(p["x"] >= x0 - tol) and np.all(p["x"] < x0 + side + tol)
            assert np.all(p["y"] >= y0 - tol) and np.all(p["y"] < y0 + side + tol)
            assert np.array_equal(np.bincount(leaf, minlength=M.nleaf).astype(np.float64), counts[s])
            assert np.unique(p["id"]).size == p["id"].size
            charge += cfg["q"][s] * p["w"].sum()
            scale += abs(cfg["q"][s]) * p["w"].sum()
            idx = rng.choice(p["x"].size, 20_000, replace=False)
            sample[s] = {k: np.ascontiguousarray(v[idx]) for k, v in p.items()}
            del p, leaf, x0, y0, side
        # the deposit: sum over leaves of rho * area is the total charge
        area = (M.s * hf) ** 2
        assert abs(float((rho * area).sum()) - charge) <= 1e-9 * scale
        ctx.step(1)
        after = {}
        for s in (0, 1):
            a = ctx.particles(s)
            o = np.argsort(a["id"])
            after[s] = {k: v[o] for k, v in a.items()}
            del a
    sim = O.Sim(cfg, M)
    sim.step_count = step
    for s in (0, 1):
        smp = sample[s]
        n = smp["x"].size
        x, y = smp["x"].copy(), smp["y"].copy()
        vx, vy, vz = smp["vx"].copy(), smp["vy"].copy(), smp["vz"].copy()
        ids = smp["id"].astype(np.uint64)
        leaf = smp["leaf"].astype(np.int64)
        new_leaf = np.empty(n, np.int64)
        spawn = np.zeros(n, np.uint8)
        sv, svi = np.zeros(3 * n), np.zeros(3 * n)
        pp = sim.push_params(s)
        O.lib().or_push_mcc(C.byref(M._c), C.byref(pp), O._ptr(E), n, O._ptr(x), O._ptr(y), O._ptr(vx), O._ptr(vy),
                            O._ptr(vz), O._ptr(ids), O._ptr(leaf), O._ptr(new_leaf), O._ptr(spawn), O._ptr(sv),
                            O._ptr(svi))
        a = after[s]
        pos = np.minimum(np.searchsorted(a["id"], ids), a["id"].size - 1)
        found = a["id"][pos] == ids
        alive = new_leaf >= 0
        assert (found == alive).mean() >= 0.9995  # absorbed at a wall exactly when the oracle absorbs
        both = found & alive
        g = pos[both]
        assert both.sum() > 0.9 * n
        dx = np.maximum(np.abs(a["x"][g] - x[both]), np.abs(a["y"][g] - y[both]))
        assert np.quantile(dx, 0.999) <= 1e-5 * hf
        dv = np.sqrt((a["vx"][g] - vx[both]) ** 2 + (a["vy"][g] - vy[both]) ** 2 + (a["vz"][g] - vz[both]) ** 2)
        vmag = np.sqrt(vx[both] ** 2 + vy[both] ** 2 + vz[both] ** 2)
        assert (dv <= 1e-5 * np.maximum(vmag, 1e-3 * vmag.max())).mean() >= 0.999
        assert (a["leaf"][g].astype(np.int64) == new_leaf[both]).mean() >= 0.9999
