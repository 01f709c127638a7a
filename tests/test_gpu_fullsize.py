"""The streamer at its full size (5e7 particles, ~3.8e5 leaves after adaptation), in the launch
configuration the benchmark times: properties that hold at any size (every particle inside
the leaf that lists it, per-leaf counts, unique ids, charge conservation of the deposit), and
one step of a random sample of 200,000 particles per species recomputed by the oracle's push
and collisions from the GPU's own corner field (FP32 against FP64): a particle may differ only
when its collision decision lies inside the rounding margin (|U0 - P| <= 1e-6 P, or the process
choice within 1e-6 sigma_T of its threshold) or its new position lies within 1e-6 of its leaf
size of a face; such differences number at most 1e-5 of the sample.  Every other particle has
the oracle's absorption, leaf, position (1e-5 of the finest cell) and velocity (1e-5)."""
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
            idx = rng.choice(p["x"].size, 200_000, replace=False)
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
    n_all, disagree = 0, 0
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
        dec = np.empty(4 * n)
        pp = sim.push_params(s)
        O.lib().or_push_mcc(C.byref(M._c), C.byref(pp), O._ptr(E), n, O._ptr(x), O._ptr(y), O._ptr(vx), O._ptr(vy),
                            O._ptr(vz), O._ptr(ids), O._ptr(leaf), O._ptr(new_leaf), O._ptr(spawn), O._ptr(sv),
                            O._ptr(svi), O._ptr(dec), None)
        U0, P, U1st, siz = dec.reshape(n, 4).T
        # rounding margin of the collision decisions (FP32 against FP64 arithmetic)
        margin = (U0 >= 0) & (np.abs(U0 - P) <= 1e-6 * np.maximum(P, 1e-30))
        if s == 0:
            margin |= (U0 >= 0) & (U0 < P) & (np.abs(U1st - siz) <= 1e-6 * (cfg["sigma_el"] + siz))
        a = after[s]
        pos = np.minimum(np.searchsorted(a["id"], ids), a["id"].size - 1)
        found = a["id"][pos] == ids
        alive = new_leaf >= 0
        # ... and of the new position: within 1e-6 of the leaf size of a face (the oracle's
        # leaf, or the GPU's), which includes the walls
        def near_face(xx, yy, lf):
            ok = lf >= 0
            l2 = np.where(ok, lf, 0)
            hl = M.s[l2] * hf
            u = (xx - M.ix[l2] * hf) / hl
            v = (yy - M.iy[l2] * hf) / hl
            return ok & (np.minimum(np.minimum(u, 1 - u), np.minimum(v, 1 - v)) <= 1e-6)
        lg = np.where(found, a["leaf"][pos].astype(np.int64), -1)
        margin |= near_face(x, y, new_leaf) | near_face(a["x"][pos], a["y"][pos], lg)
        both = found & alive
        g = pos[both]
        assert both.sum() > 0.9 * n
        dx = np.maximum(np.abs(a["x"][g] - x[both]), np.abs(a["y"][g] - y[both]))
        dv = np.sqrt((a["vx"][g] - vx[both]) ** 2 + (a["vy"][g] - vy[both]) ** 2 + (a["vz"][g] - vz[both]) ** 2)
        vmag = np.sqrt(vx[both] ** 2 + vy[both] ** 2 + vz[both] ** 2)
        bad = np.zeros(n, bool)
        bad[both] = ((dx > 1e-5 * hf) | (dv > 1e-5 * np.maximum(vmag, 1e-3 * vmag.max())) |
                     (a["leaf"][g].astype(np.int64) != new_leaf[both]))
        bad |= found != alive                          # absorbed by one side only
        assert not np.any(bad & ~margin), (s, np.nonzero(bad & ~margin)[0][:10])
        disagree += int(np.count_nonzero(bad))
        n_all += n
    assert disagree <= 1e-5 * n_all, disagree
