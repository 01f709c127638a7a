"""Pins of the oracle's mesh adaptation and split/merge (§3.1, §4.3) against conservation
laws, invariants and hand-built cases (no GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_1604_07713_gb300 import workloads as W


def _streamer_sim(n=40000, nx0=16, lmax=3, precision=W.FP64, seed=1):
    tree = W.streamer_tree(nx0=nx0, lmax=lmax)
    cfg, mesh, parts = W.streamer(n_particles=n, nx0=nx0, lmax=lmax, precision=precision, tree=tree, seed=seed)
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], mesh["lmax"], cfg["bc_x"], cfg["bc_y"], mesh["root"],
               mesh["level"], mesh["morton"])
    sim = O.Sim(cfg, M)
    for s in sorted(parts):
        sim.load(s, **parts[s])
    sim.fields()
    return sim


def _totals(sim):
    out = []
    for sp in sim.species:
        out.append((sp.w.sum(), (sp.w * sp.vx).sum(), (sp.w * sp.vy).sum(), (sp.w * sp.vz).sum(),
                    (sp.w * sp.x).sum(), (sp.w * sp.y).sum()))
    return np.array(out)


def _corner_balanced(M):
    for a in range(M.nleaf):
        x, y, s = M.ix[a], M.iy[a], M.s[a]
        for (I, J) in ((x - 1, y - 1), (x + s, y - 1), (x - 1, y + s), (x + s, y + s), (x - 1, y), (x + s, y),
                       (x, y - 1), (x, y + s)):
            b = M.leaf_at(I, J)
            if b >= 0 and abs(int(M.level[a]) - int(M.level[b])) > 1:
                return False
    return True


def test_adapt_and_split_merge_conserve_charge_mass_momentum():
    sim = _streamer_sim()
    before = _totals(sim)
    st = sim.adapt()
    after = _totals(sim)
    assert st["mesh"]["coarsened"] > 0 and st["particles"]["split"] > 0 and st["particles"]["merged"] > 0
    # weight (charge, mass), momentum and charge centre (dipole) exactly up to rounding
    assert np.allclose(after, before, rtol=1e-13, atol=0)
    M = sim.mesh
    assert _corner_balanced(M)
    for sp in sim.species:
        assert np.array_equal(sp.leaf, M.locate(sp.x, sp.y, brute=True))
        assert len(set(sp.id.tolist())) == sp.n
        c = np.bincount(sp.leaf, minlength=M.nleaf)
        assert c[c > 0].min() >= sim.cfg["ppc_min"] and c.max() <= sim.cfg["ppc_max"]


def test_split_is_exact_and_merge_energy_loss_is_the_group_spread():
    cfg = W.base_config(precision=W.FP64, n_species=1, q=[-1.0], m=[2.0], bc_x=W.BC_DIRICHLET,
                        bc_y=W.BC_NEUMANN, ppc_min=8, ppc_max=128, ppc_target=32)
    M = O.Mesh(2, 1, 1.0, 0, O.BC_DIRICHLET, O.BC_NEUMANN)
    sim = O.Sim(cfg, M)
    rng = np.random.default_rng(4)
    # leaf 0: 3 particles (split twice: 3 -> 12 -> 48? no: least r with 3*4^r >= 8 is r = 1)
    # leaf 1: 200 particles (merged to 32)
    x = np.concatenate([rng.random(3) * 0.98 + 0.01, 1.0 + rng.random(200) * 0.98 + 0.01])
    y = rng.random(203) * 0.98 + 0.01
    v = rng.standard_normal((3, 203))
    w = rng.random(203) + 0.5
    sim.load(0, x, y, v[0], v[1], v[2], w)
    sp0 = sim.species[0]
    m = 2.0
    e0 = 0.5 * m * np.sum(sp0.w * (sp0.vx ** 2 + sp0.vy ** 2 + sp0.vz ** 2))
    ids0 = sp0.id.copy(); w0 = sp0.w.copy(); x0 = sp0.x.copy(); y0 = sp0.y.copy()
    vv0 = np.stack([sp0.vx, sp0.vy, sp0.vz])
    sim.adapt(mesh=False, particles=True)
    sp = sim.species[0]
    c = np.bincount(sp.leaf, minlength=2)
    assert c[0] == 12 and c[1] == 32
    # split: each parent -> 4 children of weight w/4, same velocity, charge centre at the parent
    for k in range(3):
        ch = slice(4 * k, 4 * k + 4)
        assert sp.id[4 * k] == ids0[k]
        assert np.allclose(sp.w[ch], w0[k] / 4, rtol=0, atol=1e-15)
        assert np.allclose(np.sum(sp.w[ch] * sp.x[ch]) / w0[k], x0[k], rtol=0, atol=1e-15)
        assert np.allclose(np.sum(sp.w[ch] * sp.y[ch]) / w0[k], y0[k], rtol=0, atol=1e-15)
        assert np.all(sp.vx[ch] == vv0[0, k])
    # new ids: next_id onwards, in list order
    assert sorted(sp.id[np.isin(sp.id, ids0, invert=True)].tolist()) == list(range(203, 203 + 9))
    # merge: kinetic energy lost = sum over groups of the weighted velocity spread
    e1 = 0.5 * m * np.sum(sp.w * (sp.vx ** 2 + sp.vy ** 2 + sp.vz ** 2))
    bins = O.adapt._energy_bins(vv0[0, 3:], vv0[1, 3:], vv0[2, 3:], 0.5 * m, fp32=False)
    order = np.lexsort((ids0[3:], bins))
    q, r = divmod(200, 32)
    pos, loss = 0, 0.0
    for g in range(32):
        size = q + 1 if g < r else q
        idx = 3 + order[pos:pos + size]
        pos += size
        W_ = w0[idx].sum()
        V = (w0[idx] * vv0[:, idx]).sum(axis=1) / W_
        loss += 0.5 * m * np.sum(w0[idx] * ((vv0[:, idx] - V[:, None]) ** 2).sum(axis=0))
    assert abs((e0 - e1) - loss) < 1e-12 * e0


def test_merge_with_at_most_twice_the_target_is_pairwise():
    cfg = W.base_config(precision=W.FP64, n_species=1, q=[-1.0], m=[1.0], bc_x=W.BC_DIRICHLET,
                        bc_y=W.BC_NEUMANN, ppc_min=8, ppc_max=36, ppc_target=32)
    M = O.Mesh(1, 1, 1.0, 0, O.BC_DIRICHLET, O.BC_NEUMANN)
    sim = O.Sim(cfg, M)
    rng = np.random.default_rng(2)
    n = 40
    x = rng.random(n) * 0.9 + 0.05; y = rng.random(n) * 0.9 + 0.05
    v = rng.standard_normal((3, n)); w = np.ones(n)
    sim.load(0, x, y, v[0], v[1], v[2], w)
    sim.adapt(mesh=False, particles=True)
    sp = sim.species[0]
    assert sp.n == 32
    bins = O.adapt._energy_bins(v[0], v[1], v[2], 0.5, fp32=False)
    order = np.lexsort((np.arange(n), bins))
    # first 8 outputs: pairs (1st+2nd), (3rd+4th), ... of the sorted list; then 24 singles
    for g in range(8):
        a, b = order[2 * g], order[2 * g + 1]
        assert abs(sp.vx[g] - 0.5 * (v[0, a] + v[0, b])) < 1e-15
        assert sp.id[g] == min(a, b)
    assert np.array_equal(sp.id[8:], order[16:].astype(np.uint64))


def test_refinement_by_count_hands_particles_to_children_and_keeps_phi():
    cfg = W.base_config(precision=W.FP64, n_species=1, q=[-1.0], m=[1.0], bc_x=W.BC_DIRICHLET,
                        bc_y=W.BC_NEUMANN, max_level=2, refine_count=50, coarsen_count=-1,
                        e_ref=1e30, phi_right=1.0)
    M = O.Mesh(4, 4, 0.25, 2, O.BC_DIRICHLET, O.BC_NEUMANN)
    sim = O.Sim(cfg, M)
    rng = np.random.default_rng(8)
    # 80 particles in root 5 (x in [0.25,0.5), y in [0.25,0.5)), 10 elsewhere
    x = np.concatenate([0.25 + 0.25 * rng.random(80), rng.random(10)])
    y = np.concatenate([0.25 + 0.25 * rng.random(80), 0.5 + 0.5 * rng.random(10)])
    z = np.zeros(90)
    sim.load(0, x, y, z, z, z, np.full(90, 1e-9))
    sim.fields()
    phi_before = sim.phi.copy()
    st = sim.adapt(particles=False)["mesh"]
    M2 = sim.mesh
    assert st["refined"] == 1 and M2.nleaf == 16 + 3
    kids = np.nonzero(M2.level == 1)[0]
    assert len(kids) == 4 and np.all(M2.root[kids] == 5)
    assert np.allclose(sim.phi[kids], phi_before[5])
    sp = sim.species[0]
    assert np.array_equal(sp.leaf, M2.locate(sp.x, sp.y, brute=True))
    assert np.bincount(sp.leaf, minlength=M2.nleaf)[kids].sum() == 80


def test_balance_closure_refines_neighbours_of_deep_refinement():
    # a level-2 region next to level-0 leaves: refining a level-2 leaf to 3 forces the chain
    r, l, m = W.region_tree(4, 4, 2, lambda lv, xc, yc, h: abs(xc / 4 - 0.4) < 0.2 and abs(yc / 4 - 0.4) < 0.2)
    cfg = W.base_config(precision=W.FP64, n_species=1, q=[-1.0], m=[1.0], bc_x=W.BC_DIRICHLET,
                        bc_y=W.BC_NEUMANN, max_level=3, refine_count=20, coarsen_count=-1, e_ref=1e30)
    M = O.Mesh(4, 4, 0.25, 3, O.BC_DIRICHLET, O.BC_NEUMANN, r, l, m)
    sim = O.Sim(cfg, M)
    deep = np.nonzero(M.level == M.level.max())[0][0]
    h = M.s[deep] * M.hf
    rng = np.random.default_rng(1)
    x = M.ix[deep] * M.hf + h * (0.05 + 0.9 * rng.random(30))
    y = M.iy[deep] * M.hf + h * (0.05 + 0.9 * rng.random(30))
    z = np.zeros(30)
    sim.load(0, x, y, z, z, z, np.full(30, 1e-9))
    sim.fields()
    sim.adapt(particles=False)
    assert sim.mesh.level.max() == M.level.max() + 1
    assert _corner_balanced(sim.mesh)


def test_field_criterion_alone_refines_and_blocks_coarsening_hand_case():
    """No particles, so the count criterion never fires; the potential depends on x only and
    its face gradients are written out by hand.  8 x 4 roots of side 1, Dirichlet in x
    (phi = 0 and 14 on the walls), Neumann in y; cell-centred phi per column
    0.5, 1.5, 2.5, 3.5, 7.5, 11.5, 12.5, 13.5: face gradients 1 (wall), 1, 1, 1, 4, 4, 1, 1,
    1 (wall), so the centre |E| of the columns is 1, 1, 1, 2.5, 4, 2.5, 1, 1.  With
    e_ref = 2 and refine_field = 0.75 (threshold 1.5) exactly the 12 leaves of columns 3-5
    refine.  Second case: every root refined once, fine-column gradients 1 except 1.3 on the
    two faces of fine column 8, so only that column's |E| (1.3) reaches coarsen_field
    e_ref = 1.2: its four quartets stay fine and the other 28 coarsen.  Fails for: the
    threshold taken without e_ref, the coarsening test against refine_field, or the field
    criterion read from the corner field instead of the centre."""
    cfg = W.base_config(precision=W.FP64, n_species=1, q=[-1.0], m=[1.0], bc_x=W.BC_DIRICHLET,
                        bc_y=W.BC_NEUMANN, max_level=1, refine_count=128, coarsen_count=32,
                        e_ref=2.0, refine_field=0.75, coarsen_field=0.6)
    M = O.Mesh(8, 4, 1.0, 1, O.BC_DIRICHLET, O.BC_NEUMANN)
    sim = O.Sim(cfg, M)
    col = M.ix >> 1
    phi_col = np.array([0.5, 1.5, 2.5, 3.5, 7.5, 11.5, 12.5, 13.5])
    sim.phi = phi_col[col]
    sim.last_walls = np.array([0.0, 14.0, 0.0, 0.0])
    emag = M.cell_emag(sim.phi, sim.last_walls)
    assert np.abs(emag - np.array([1, 1, 1, 2.5, 4, 2.5, 1, 1])[col]).max() < 1e-14
    st = sim.adapt(particles=False)["mesh"]
    M2 = sim.mesh
    assert st["refined"] == 12 and st["coarsened"] == 0 and M2.nleaf == 32 - 12 + 48
    fine_roots = np.unique(M2.root[M2.level == 1])
    assert sorted((fine_roots % 8).tolist()) == [3, 3, 3, 3, 4, 4, 4, 4, 5, 5, 5, 5]

    # every root refined once: 16 x 8 fine leaves of side 1/2
    r, l, m = W.region_tree(8, 4, 1, lambda lv, xc, yc, h: True)
    M = O.Mesh(8, 4, 1.0, 1, O.BC_DIRICHLET, O.BC_NEUMANN, r, l, m)
    cfg["e_ref"] = 1.0
    cfg["coarsen_field"] = 1.2
    sim = O.Sim(cfg, M)
    fcol = M.ix                                   # fine column 0..15
    g = np.ones(17)                               # gradients of faces 0..16 (0, 16: walls)
    g[8] = g[9] = 1.3                             # the two faces of fine column 8
    # phi at fine-column centres from the face gradients (h = 1/2; the wall face is h/4 away)
    phi_f = np.empty(16)
    phi_f[0] = g[0] * 0.25
    for j in range(1, 16):
        phi_f[j] = phi_f[j - 1] + g[j] * 0.5
    sim.phi = phi_f[fcol]
    sim.last_walls = np.array([0.0, phi_f[15] + g[16] * 0.25, 0.0, 0.0])
    emag = M.cell_emag(sim.phi, sim.last_walls)
    expect = np.where(fcol == 8, 1.3, np.where((fcol == 7) | (fcol == 9), 1.15, 1.0))
    assert np.abs(emag - expect).max() < 1e-12
    st = sim.adapt(particles=False)["mesh"]
    M2 = sim.mesh
    assert st["refined"] == 0 and st["coarsened"] == 28 and M2.nleaf == 28 + 16
    assert np.all((M2.root[M2.level == 1] % 8) == 4)
