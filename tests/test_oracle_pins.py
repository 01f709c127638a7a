"""Pins of the FP64 oracle against facts fixed by the paper, by mathematics or by
independent brute force (no GPU).  Each test names the part of the method it pins."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1604_07713_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11): published known-answer vectors + invertibility
# --------------------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox(np.array([v[0]], np.uint32), v[1], v[2], v[3], v[4], v[5])[0]
        assert list(map(int, out)) == v[6:10]


def test_philox_round_structure_is_invertible():
    # The Philox S-box is a bijection: multipliers are odd, so each round can be undone with
    # their inverses mod 2^32.  Inverting ten rounds must give back the counter.
    M0, M1 = 0xD2511F53, 0xCD9E8D57
    W0, W1 = 0x9E3779B9, 0xBB67AE85
    inv0, inv1 = pow(M0, -1, 1 << 32), pow(M1, -1, 1 << 32)
    rng = np.random.default_rng(1)
    for _ in range(20):
        c = [int(t) for t in rng.integers(0, 1 << 32, 4, dtype=np.uint64)]
        k = [int(t) for t in rng.integers(0, 1 << 32, 2, dtype=np.uint64)]
        out = [int(t) for t in O.philox(np.array([c[0]], np.uint32), c[1], c[2], c[3], k[0], k[1])[0]]
        x = out
        for r in range(9, -1, -1):
            k0 = (k[0] + r * W0) & 0xFFFFFFFF
            k1 = (k[1] + r * W1) & 0xFFFFFFFF
            lo0, lo1 = x[3], x[1]
            c0 = (lo0 * inv0) & 0xFFFFFFFF
            c2 = (lo1 * inv1) & 0xFFFFFFFF
            hi0 = (M0 * c0) >> 32
            hi1 = (M1 * c2) >> 32
            c1 = x[0] ^ hi1 ^ k0
            c3 = x[2] ^ hi0 ^ k1
            x = [c0, c1, c2, c3]
        assert x == c


def test_philox_uniformity_and_exact_uniforms():
    from scipy import stats
    n = 1 << 18
    r = O.philox(np.arange(n, dtype=np.uint32), 7, 11, 0, 0x12345678, 0x9ABCDEF0)
    u = O.uniform24(r.reshape(-1))
    assert np.all(u.astype(np.float32).astype(np.float64) == u)  # exact in FP32
    assert u.min() >= 0.0 and u.max() < 1.0
    counts = np.bincount((u * 256).astype(int), minlength=256)
    p = stats.chisquare(counts).pvalue
    assert 1e-5 < p < 1 - 1e-5
    # the four lanes are uncorrelated
    U = O.uniform24(r)
    cc = np.corrcoef(U.T)
    assert np.abs(cc - np.eye(4)).max() < 0.01


# --------------------------------------------------------------------------------------
# Morton order and the leaf tree (§2.1 SFC, §3.1 quadtree)
# --------------------------------------------------------------------------------------
def test_morton_closed_form():
    assert [O.morton(x, y) for x, y in [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (3, 3)]] == \
        [0, 1, 2, 3, 4, 8, 15]
    for x in range(16):
        for y in range(16):
            m = O.morton(x, y)
            assert sum(((m >> (2 * b)) & 1) << b for b in range(8)) == x
            assert sum(((m >> (2 * b + 1)) & 1) << b for b in range(8)) == y


@pytest.mark.parametrize("seed,px,py", [(1, False, True), (2, True, True), (3, False, False)])
def test_tree_tiling_balance_and_bruteforce_locate(seed, px, py):
    nx0, ny0, lmax = 3, 2, 4
    r, l, m = W.random_tree(nx0, ny0, lmax, 0.35, seed, px, py)
    bcx = O.BC_PERIODIC if px else O.BC_DIRICHLET
    bcy = O.BC_PERIODIC if py else O.BC_NEUMANN
    M = O.Mesh(nx0, ny0, 0.5, lmax, bcx, bcy, r, l, m)
    assert M.nleaf <= 256 * 4
    # leaves tile the domain exactly
    assert np.isclose(M.area().sum(), M.lx * M.ly, rtol=0, atol=1e-15)
    # random points, plus points exactly on faces and corners (dyadic h0 -> exact floats)
    rng = np.random.default_rng(seed)
    xs = rng.random(3000) * M.lx; ys = rng.random(3000) * M.ly
    xf = M.ix * M.hf; yf = M.iy * M.hf
    xs = np.concatenate([xs, xf, xf + 0.5 * M.h(), xf]); ys = np.concatenate([ys, yf, yf, yf + 0.5 * M.h()])
    a = M.locate(xs, ys)
    b = M.locate(xs, ys, brute=True)
    assert np.array_equal(a, b)
    # face neighbours are symmetric: if B is across A's face d, A is across B's opposite face
    t, n1, n2, sib = M.face_table()
    opp = [1, 0, 3, 2]
    for A in range(M.nleaf):
        for d in range(4):
            if t[A, d] == 1:
                assert t[n1[A, d], opp[d]] == 1 and n1[n1[A, d], opp[d]] == A
            elif t[A, d] == 3:
                for B in (n1[A, d], n2[A, d]):
                    assert t[B, opp[d]] == 2 and n1[B, opp[d]] == A


# --------------------------------------------------------------------------------------
# Poisson on the composite leaf mesh (§3: multigrid Poisson, potential at cell centres)
# --------------------------------------------------------------------------------------
def _disk_tree(n, lmax):
    return W.region_tree(n, n, lmax, lambda lv, xc, yc, h: (xc / n - 0.5) ** 2 + (yc / n - 0.5) ** 2 < 0.09)


def test_linear_potential_and_uniform_field_exact_on_amr():
    n = 8
    r, l, m = _disk_tree(n, 3)
    M = O.Mesh(n, n, 1.0 / n, 3, O.BC_DIRICHLET, O.BC_NEUMANN, r, l, m)
    assert len(np.unique(M.s)) == 4
    xc, _ = M.centres()
    walls = [0.0, 2.5, 0.0, 0.0]
    phi = M.solve_poisson(np.zeros(M.nleaf), walls)
    assert np.abs(phi - 2.5 * xc).max() < 1e-13
    E = M.node_e(phi, walls)  # uniform field E = -2.5 x, exact at every corner incl. hanging nodes
    assert np.abs(E[:, :, 0] + 2.5).max() < 1e-12 and np.abs(E[:, :, 1]).max() < 1e-12


def _mms_errors(amr):
    errs = []
    for n in (16, 32, 64):
        if amr:
            r, l, m = _disk_tree(n, 2)
            M = O.Mesh(n, n, 1.0 / n, 2, O.BC_DIRICHLET, O.BC_DIRICHLET, r, l, m)
        else:
            M = O.Mesh(n, n, 1.0 / n, 0, O.BC_DIRICHLET, O.BC_DIRICHLET)
        xc, yc = M.centres(); h = M.h()
        f = 2 * np.pi ** 2 * np.sin(np.pi * xc) * np.sin(np.pi * yc)
        phi = M.solve_poisson(f * h * h, [0, 0, 0, 0])
        e = phi - np.sin(np.pi * xc) * np.sin(np.pi * yc)
        errs.append((np.sqrt((e * e * h * h).sum()), np.abs(e).max()))
    return np.array(errs)


@pytest.mark.parametrize("amr", [False, True])
def test_poisson_second_order_manufactured_solution(amr):
    e = _mms_errors(amr)
    order = np.log2(e[:-1] / e[1:])
    assert order[:, 0].min() >= 1.8, order   # L2
    assert order[-1, 1] >= 1.8, order        # max norm on the finest pair


def test_poisson_periodic_equals_fft_eigen_solve():
    n = 32
    M = O.Mesh(n, n, 1.0 / n, 0, O.BC_PERIODIC, O.BC_PERIODIC)
    rng = np.random.default_rng(5)
    rho = rng.standard_normal(M.nleaf); rho -= rho.mean()
    h = M.h()[0]
    phi = M.solve_poisson(rho * h * h, [0, 0, 0, 0])
    # 5-point Laplacian eigenvalues on the periodic lattice; leaves are in Morton order
    grid = np.zeros((n, n)); grid[M.iy, M.ix] = rho
    k = np.fft.fftfreq(n) * n
    lam = (4 * np.sin(np.pi * k / n) ** 2)[None, :] + (4 * np.sin(np.pi * k / n) ** 2)[:, None]
    lam[0, 0] = 1.0
    F = np.fft.fft2(grid * h * h) / lam; F[0, 0] = 0.0
    ref = np.real(np.fft.ifft2(F))
    assert np.abs(phi - ref[M.iy, M.ix]).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_operator_is_conservative():
    r, l, m = W.random_tree(4, 4, 3, 0.3, 9, True, True)
    M = O.Mesh(4, 4, 0.25, 3, O.BC_PERIODIC, O.BC_PERIODIC, r, l, m)
    A, _ = M.operator()
    # fluxes cancel pairwise: every column of the integrated operator sums to zero
    assert np.abs(np.asarray(A.sum(axis=0))).max() < 1e-14


# --------------------------------------------------------------------------------------
# Deposit, push, cell lists (§3 NGP + leapfrog, §3.1 cell-based lists)
# --------------------------------------------------------------------------------------
def test_single_particle_in_uniform_field_exact_leapfrog():
    # plates at x = 0 (0 V) and x = 1 (V0), no charge: E = -V0 x-hat everywhere, on an AMR tree
    n, lmax = 8, 2
    r, l, m = _disk_tree(n, lmax)
    mesh = dict(nx0=n, ny0=n, h0=1.0 / n, lmax=lmax)
    cfg = W.base_config(precision=W.FP64, n_species=1, dt=0.01, eps0=1.0, q=[2.0], m=[4.0],
                        bc_x=W.BC_DIRICHLET, bc_y=W.BC_NEUMANN, phi_right=3.0)
    M = O.Mesh(n, n, 1.0 / n, lmax, O.BC_DIRICHLET, O.BC_NEUMANN, r, l, m)
    sim = O.Sim(cfg, M)
    sim.load(0, [0.9], [0.37], [-0.5], [0.2], [0.1], [0.0])  # weight 0: no charge
    x0, y0, v0 = 0.9, 0.37, np.array([-0.5, 0.2])
    a = 2.0 / 4.0 * (-3.0)
    for k in range(1, 31):
        sim.step()
        sp = sim.species[0]
        vx = -0.5 + a * 0.01 * k
        assert abs(sp.vx[0] - vx) < 1e-13 and abs(sp.vy[0] - 0.2) < 1e-13 and sp.vz[0] == 0.1
        # x^k = x0 + sum_j v^{j+1/2} dt : quadratic in k
        xk = x0 + 0.01 * (-0.5 * k + a * 0.01 * k * (k + 1) / 2)
        assert abs(sp.x[0] - xk) < 1e-13 and abs(sp.y[0] - (y0 + 0.2 * 0.01 * k)) < 1e-13
        assert sp.leaf[0] == M.locate(sp.x, sp.y)[0]


def test_deposit_conserves_charge_and_cell_lists_are_consistent():
    cfg, mesh, parts = W.ccp(nx=32, ny=4, ppc=20, seed=3, precision=W.FP64)
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], 0, O.BC_DIRICHLET, O.BC_PERIODIC)
    sim = O.Sim(cfg, M)
    for s in (0, 1):
        sim.load(s, **parts[s])
    Q = sim.charge()
    tot = sum(sp.q * sp.w.sum() for sp in sim.species)
    assert abs(Q.sum() - tot) <= 1e-12 * sum(abs(sp.q) * sp.w.sum() for sp in sim.species)
    for _ in range(5):
        ids_before = [set(sp.id.tolist()) for sp in sim.species]
        sim.step()
        for s, sp in enumerate(sim.species):
            assert np.all(np.diff(sp.leaf) >= 0)                  # lists in leaf order
            assert np.array_equal(sp.leaf, M.locate(sp.x, sp.y))  # every particle in its leaf
            assert len(set(sp.id.tolist())) == sp.n               # ids unique
            new = set(sp.id.tolist()) - ids_before[s]
            assert all(i >= min(new) for i in new) if new else True


def test_cell_list_order_rule():
    # stayers keep their order at the head of each list; entering particles are appended in
    # the order of their old list position
    sp = O.Species(-1.0, 1.0, *[np.zeros(6) for _ in range(6)],
                   np.arange(6, dtype=np.uint64), np.array([0, 0, 1, 1, 2, 2]))
    new_leaf = np.array([1, 0, 1, 0, -1, 2])
    out = O.Sim._rebin(sp, new_leaf, None)
    assert out.leaf.tolist() == [0, 0, 1, 1, 2]
    assert out.id.tolist() == [1, 3, 2, 0, 5]


# --------------------------------------------------------------------------------------
# Monte Carlo collisions (§3 MCC): binomial collision count, branching, energy loss
# --------------------------------------------------------------------------------------
def _mcc_sim(n, speed, sig_el, sig_iz, eps_th, ng, dt, ions=False):
    mesh = O.Mesh(4, 4, 0.25, 0, O.BC_PERIODIC, O.BC_PERIODIC)
    cfg = W.base_config(precision=W.FP64, n_species=2, dt=dt, eps0=1.0, q=[-W.QE, W.QE],
                        m=[W.ME, 4 * W.AMU], qe=W.QE, mcc=1, gas_density=ng,
                        gas_temperature_ev=0.0 if not ions else 0.026, neutral_mass=4 * W.AMU,
                        sigma_el=sig_el, sigma_iz0=sig_iz, eps_th_ev=eps_th)
    sim = O.Sim(cfg, mesh)
    rng = np.random.default_rng(0)
    x = rng.random(n); y = rng.random(n)
    d = rng.standard_normal((3, n)); d /= np.linalg.norm(d, axis=0)
    s = 0 if not ions else 1
    sim.load(0, x[:0], y[:0], x[:0], x[:0], x[:0], x[:0]) if ions else None
    sim.load(s, x, y, speed * d[0], speed * d[1], speed * d[2], np.zeros(n))
    if not ions:
        sim.load(1, x[:0], y[:0], x[:0], x[:0], x[:0], x[:0])
    return sim


def test_mcc_collision_count_is_binomial_and_branching_matches_cross_sections():
    n = 200_000
    eps = 60.0
    speed = np.sqrt(2 * eps * W.QE / W.ME)
    sig_el, sig0, th = 6e-20, 1e-20, 24.6
    ng, dt = 1e21, 2e-12
    sim = _mcc_sim(n, speed, sig_el, sig0, th, ng, dt)
    before = sim.species[0].vx.copy()
    sim.step()
    sp = sim.species[0]
    siz = sig0 * (1 - th / eps)
    P = 1 - np.exp(-ng * (sig_el + siz) * speed * dt)
    n_iz = sim.species[1].n
    # collided = ionized parents + elastically scattered (speed changed or direction changed)
    par = sp.id < n
    sp_speed = np.sqrt(sp.vx ** 2 + sp.vy ** 2 + sp.vz ** 2)[par]
    collided = np.count_nonzero(np.abs(sp_speed - speed) > 1e-9 * speed)
    mean, sd = n * P, np.sqrt(n * P * (1 - P))
    assert abs(collided - mean) < 5 * sd, (collided, mean, sd)
    frac = siz / (sig_el + siz)
    assert abs(n_iz - collided * frac) < 5 * np.sqrt(collided * frac * (1 - frac))
    # ionization conserves energy: e1 + e2 = eps - eps_th for every pair
    assert sim.species[0].n == n + n_iz


def test_mcc_elastic_mean_energy_loss_is_2m_over_M():
    n = 400_000
    eps = 10.0
    speed = np.sqrt(2 * eps * W.QE / W.ME)
    sim = _mcc_sim(n, speed, 6e-20, 0.0, 24.6, 1e22, 1e-11)
    sim.step()
    sp = sim.species[0]
    e_after = 0.5 * W.ME * (sp.vx ** 2 + sp.vy ** 2 + sp.vz ** 2) / W.QE
    hit = np.abs(e_after - eps) > 1e-9 * eps
    loss = (eps - e_after[hit]).mean() / eps
    expect = 2 * W.ME / (4 * W.AMU)  # isotropic: <1 - cos chi> = 1
    assert abs(loss - expect) < 0.02 * expect


# --------------------------------------------------------------------------------------
# Whole cycle: cold-plasma oscillation at omega_p, energy conservation
# --------------------------------------------------------------------------------------
@pytest.mark.slow
def test_cold_plasma_oscillates_at_plasma_frequency():
    # Quiet start (regular sub-lattice) so that only the seeded k = 2 pi mode is present;
    # amplitude 20 % so that NGP sees the sheet displacement (still below sheet crossing, so
    # the cold-plasma oscillation is exactly linear at omega = omega_p = 1).
    cfg, mesh, parts = W.cold_plasma(n_side=64, ppc=16, dt=0.05, quiet=True, amp=0.2)
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], 0, O.BC_PERIODIC, O.BC_PERIODIC)
    sim = O.Sim(cfg, M)
    sim.load(0, **parts[0])
    xc, _ = M.centres()
    We, Ke, mode = [], [], []
    for _ in range(200):
        vprev = dict(zip(sim.species[0].id.tolist(), zip(sim.species[0].vx, sim.species[0].vy)))
        sim.step()
        rho, phi, E = sim.last_rho, sim.phi, sim.last_node_e
        We.append(0.5 * np.sum(rho * phi * M.area()))
        mode.append(np.sum(E[:, 0, 0] * np.sin(2 * np.pi * xc)))
        sp = sim.species[0]
        pv = np.array([vprev[i] for i in sp.id.tolist()])
        # kinetic energy at integer time from the two half-step velocities
        Ke.append(0.5 * np.sum(sp.w * (pv[:, 0] * sp.vx + pv[:, 1] * sp.vy)))
    We, Ke, mode = np.array(We), np.array(Ke), np.array(mode)
    t = np.arange(200) * 0.05
    # least-squares frequency of the k = 2 pi field mode
    ws = np.linspace(0.8, 1.2, 4001)
    res = []
    for w in ws:
        B = np.stack([np.cos(w * t), np.sin(w * t)], 1)
        c = np.linalg.lstsq(B, mode, rcond=None)[0]
        res.append(np.sum((B @ c - mode) ** 2))
    w_fit = ws[int(np.argmin(res))]
    assert abs(w_fit - 1.0) < 0.01, w_fit
    # NGP (momentum-conserving) is not exactly energy-conserving: the total fluctuates as
    # sheets cross cell faces, but shows no secular drift over the run
    tot = We + Ke
    per = int(round(np.pi / 0.05))
    assert abs(tot[-per:].mean() - tot[:per].mean()) < 0.01 * We.max()
    assert (tot.max() - tot.min()) < 0.1 * We.max()
