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


def test_philox2x32_known_answers():
    # the collision test's uniform comes from the 2x32 form
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox2x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert O.philox2(v[0], v[1], v[2]) == (v[3], v[4])


def test_philox2x32_round_structure_is_invertible():
    # one odd multiplier: each round is undone with its inverse mod 2^32
    M, W_ = 0xD256D193, 0x9E3779B9
    inv = pow(M, -1, 1 << 32)
    rng = np.random.default_rng(2)
    for _ in range(20):
        c0, c1, k = (int(t) for t in rng.integers(0, 1 << 32, 3, dtype=np.uint64))
        x0, x1 = O.philox2(c0, c1, k)
        for r in range(9, -1, -1):
            kr = (k + r * W_) & 0xFFFFFFFF
            p0 = (x1 * inv) & 0xFFFFFFFF       # the round's input word 0
            hi = (M * p0) >> 32
            x0, x1 = p0, x0 ^ hi ^ kr           # and word 1
        assert (x0, x1) == (c0, c1)


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


def test_periodic_wrap_is_modulo_the_period():
    """A particle that moves 2.3 periods in a periodic direction in one step ends at its
    position modulo the period (and keeps its velocity); one that leaves through an
    absorbing wall is removed.  Fails for: a single wrap (the particle would end outside the
    domain or be clamped to the wall)."""
    M = O.Mesh(4, 2, 0.25, 0, O.BC_DIRICHLET, O.BC_PERIODIC)
    cfg = W.base_config(precision=W.FP64, n_species=1, dt=1.0, eps0=1.0, q=[-1.0], m=[1.0],
                        bc_x=W.BC_DIRICHLET, bc_y=W.BC_PERIODIC)
    sim = O.Sim(cfg, M)
    sim.load(0, [0.3, 0.6, 0.9], [0.1, 0.2, 0.3], [0.0, 0.0, 0.5], [2.3 * 0.5, -2.3 * 0.5, 0.0],
             [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    sim.step(1)
    sp = sim.species[0]
    assert sp.n == 2                                    # the third left through x = 1
    o = np.argsort(sp.id)
    assert np.allclose(sp.y[o], [(0.1 + 1.15) % 0.5, (0.2 - 1.15) % 0.5], atol=1e-15)
    assert np.allclose(sp.x[o], [0.3, 0.6]) and np.allclose(sp.vy[o], [1.15, -1.15])
    assert np.array_equal(sp.leaf, M.locate(sp.x, sp.y))


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
    # every ionization adds one electron (its energy split is pinned below)
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


# --------------------------------------------------------------------------------------
# Direct implicit PIC (§3 DIPIC): the susceptibility operator and the implicit push
# --------------------------------------------------------------------------------------
def test_kappa_operator_special_cases_and_conservation():
    r, l, m = W.random_tree(4, 4, 3, 0.3, 9, True, True)
    M = O.Mesh(4, 4, 0.25, 3, O.BC_PERIODIC, O.BC_PERIODIC, r, l, m)
    A, _ = M.operator()
    # kappa = 1 is the explicit operator, a constant kappa scales it
    A1, _ = M.operator_kappa(np.ones(M.nleaf))
    assert abs(A1 - A).max() < 1e-15
    A3, _ = M.operator_kappa(np.full(M.nleaf, 3.0))
    assert abs(A3 - 3.0 * A).max() < 1e-14
    # a varying kappa keeps the fluxes pairwise equal and opposite (columns sum to zero) and
    # the operator as symmetric as the explicit one
    kap = 1.0 + np.random.default_rng(4).random(M.nleaf) * 5.0
    Ak, _ = M.operator_kappa(kap)
    assert np.abs(np.asarray(Ak.sum(axis=0))).max() < 1e-13
    assert abs(Ak - Ak.T).max() <= 10.0 * abs(A - A.T).max() + 1e-13
    # Dirichlet walls: the wall coefficient is the wall cell's kappa times 2
    M2 = O.Mesh(4, 2, 0.25, 0, O.BC_DIRICHLET, O.BC_PERIODIC)
    kap2 = np.arange(1.0, M2.nleaf + 1.0)
    _, bc = M2.operator_kappa(kap2)
    _, bc1 = M2.operator()
    assert np.array_equal(bc, bc1 * kap2[:, None])


def test_kappa_operator_two_cell_hand_case():
    # 2 x 1 cells, Dirichlet in x, Neumann in y: rows (2 k0 + (k0 + k1)/2, -(k0 + k1)/2),
    # (-(k0 + k1)/2, (k0 + k1)/2 + 2 k1)
    M = O.Mesh(2, 1, 0.5, 0, O.BC_DIRICHLET, O.BC_NEUMANN)
    A, bc = M.operator_kappa(np.array([2.0, 6.0]))
    assert np.allclose(A.toarray(), [[4.0 + 4.0, -4.0], [-4.0, 4.0 + 12.0]], rtol=0, atol=1e-15)
    assert np.allclose(bc, [[4.0, 0, 0, 0], [0, 12.0, 0, 0]], rtol=0, atol=1e-15)


def _implicit_mode_series(dt, nsteps, implicit=1):
    cfg, mesh, parts = W.cold_plasma(n_side=64, ppc=16, dt=dt, quiet=True, amp=0.2)
    cfg["implicit"] = implicit
    M = O.Mesh(mesh["nx0"], mesh["ny0"], mesh["h0"], 0, O.BC_PERIODIC, O.BC_PERIODIC)
    sim = O.Sim(cfg, M)
    sim.load(0, **parts[0])
    xc, _ = M.centres()
    mode = []
    for _ in range(nsteps):
        sim.step()
        mode.append(np.sum(sim.last_node_e[:, 0, 0] * np.sin(2 * np.pi * xc)))
    return np.array(mode)


def test_implicit_cold_plasma_follows_the_schemes_discrete_dispersion():
    # The implicit scheme v' = v + dt a(x'), x' = x + dt v' applied to a cold plasma mode of
    # frequency w: x_{n+1} (1 + w^2 dt^2) - 2 x_n + x_{n-1} = 0, so the mode obeys
    # m_{n+1} = a m_n + b m_{n-1} with a = 2 / (1 + W), b = -1 / (1 + W), W = (w dt)^2:
    # damped by 1 / sqrt(1 + W) per step at the phase atan(w dt) -- stable at any dt.
    # A factor 1/2 in the susceptibility, or the field without it, gives other (a, b).
    for dt, n in ((0.5, 12),):
        m = _implicit_mode_series(dt, n)
        a, b = np.linalg.lstsq(np.stack([m[1:-1], m[:-2]], 1), m[2:], rcond=None)[0]
        W_ = dt * dt  # omega_p = 1 in these units
        assert abs(a - 2.0 / (1.0 + W_)) < 0.01 and abs(b + 1.0 / (1.0 + W_)) < 0.01, (a, b)


def test_implicit_scheme_is_stable_beyond_the_explicit_limit():
    # omega_p dt = 2.5 > 2: the leapfrog mode grows, the implicit one decays
    # (until the leapfrog's sheets cross; the implicit mode decays to the NGP noise floor)
    imp = _implicit_mode_series(2.5, 8)
    exp_ = _implicit_mode_series(2.5, 8, implicit=0)
    assert np.abs(imp[3:]).max() < 0.1 * abs(imp[0])
    assert np.abs(exp_).max() > 4.0 * abs(exp_[0])


# --------------------------------------------------------------------------------------
# Ion collisions (§3 MCC of ions with neutrals): a Maxwellian neutral partner, isotropic
# scattering in the centre-of-mass frame
# --------------------------------------------------------------------------------------
def _ion_sim(n, speed, ng, dt, t_gas, m_ion, m_neutral, sig=6e-20, seed=0):
    mesh = O.Mesh(4, 4, 0.25, 0, O.BC_PERIODIC, O.BC_PERIODIC)
    cfg = W.base_config(precision=W.FP64, n_species=2, dt=dt, eps0=1.0, q=[-W.QE, W.QE],
                        m=[W.ME, m_ion], qe=W.QE, mcc=1, gas_density=ng, gas_temperature_ev=t_gas,
                        neutral_mass=m_neutral, sigma_el=sig, sigma_iz0=0.0, eps_th_ev=24.6)
    sim = O.Sim(cfg, mesh)
    rng = np.random.default_rng(seed)
    x = rng.random(n); y = rng.random(n)
    d = rng.standard_normal((3, n)); d /= np.linalg.norm(d, axis=0)
    sim.load(0, x[:0], y[:0], x[:0], x[:0], x[:0], x[:0])
    sim.load(1, x, y, speed * d[0], speed * d[1], speed * d[2], np.zeros(n))
    return sim


def _mean_collision_probability(k, a, vt):
    """E[1 - exp(-k g)] with g = |v - v_n|, |v| = a vt and v_n ~ Maxwellian of thermal speed
    vt (vt^2 per component): by symmetry g = vt sqrt(t + (a + z)^2), z ~ N(0, 1) along v and
    t ~ chi^2 with 2 degrees of freedom across it; Gauss-Hermite x Gauss-Laguerre quadrature."""
    zh, wh = np.polynomial.hermite_e.hermegauss(80)
    tl, wl = np.polynomial.laguerre.laggauss(80)      # int_0^inf f(s) e^{-s} ds, t = 2 s
    wh = wh / np.sqrt(2 * np.pi)
    g = vt * np.sqrt(2 * tl[None, :] + (a + zh[:, None]) ** 2)
    return float(np.sum(wh[:, None] * wl[None, :] * (1 - np.exp(-k * g))))


def test_ion_collision_count_matches_the_mean_over_the_maxwellian_partner():
    """The ion's collision probability is taken with the relative speed to a partner drawn from
    the neutral Maxwellian (thermal speed sqrt(T/M)).  The count of ions whose velocity changed
    must be binomial around N E[1 - exp(-n sigma g dt)], the expectation worked out here by
    quadrature over the Maxwellian.  Fails for: P from the ion speed alone (no partner), the
    partner drawn with the ion mass instead of the neutral mass, or a partner at rest."""
    n = 200_000
    m_ion, m_n = 4 * W.AMU, 40 * W.AMU
    t_gas = 0.5
    vt = np.sqrt(t_gas * W.QE / m_n)
    a = 1.5
    ng, sig = 1e22, 6e-20
    dt = 0.1 / (ng * sig * vt)                 # k vt = 0.1
    sim = _ion_sim(n, a * vt, ng, dt, t_gas, m_ion, m_n, sig)
    v0 = {int(i): (vx, vy, vz) for i, vx, vy, vz in zip(sim.species[1].id, sim.species[1].vx,
                                                        sim.species[1].vy, sim.species[1].vz)}
    sim.step()
    sp = sim.species[1]
    before = np.array([v0[int(i)] for i in sp.id])
    collided = np.count_nonzero(np.any(np.stack([sp.vx, sp.vy, sp.vz], 1) != before, axis=1))
    p = _mean_collision_probability(ng * sig * dt, a, vt)
    mean, sd = n * p, np.sqrt(n * p * (1 - p))
    assert abs(collided - mean) < 5 * sd, (collided, mean, sd)
    # the same count with the ion speed alone would be n (1 - exp(-k a vt)): far outside
    p_wrong = 1 - np.exp(-ng * sig * dt * a * vt)
    assert abs(n * p_wrong - mean) > 20 * sd


@pytest.mark.parametrize("m_ratio", [1.0, 10.0])
def test_ion_scatter_conserves_momentum_and_energy_of_the_pair(m_ratio):
    """Cold gas (partner at rest): after an elastic centre-of-mass scatter the neutral carries
    momentum m (v - v') and energy |m (v - v')|^2 / 2M, so every collided ion must satisfy
    m |v|^2 = m |v'|^2 + (m^2 / M) |v - v'|^2 to rounding.  Its mean retained energy fraction
    is (m^2 + M^2) / (m + M)^2 for isotropic centre-of-mass scattering.  Fails for: an
    isotropic scatter in the lab frame, the reduced-mass factor M/(m+M) swapped for m/(m+M),
    or the centre-of-mass velocity weighted by the wrong masses."""
    n = 100_000
    m_ion = 4 * W.AMU
    m_n = m_ratio * m_ion
    speed = 2.0e4
    ng, sig = 1e22, 6e-20
    dt = 0.5 / (ng * sig * speed)
    sim = _ion_sim(n, speed, ng, dt, 0.0, m_ion, m_n, sig)
    v0 = {int(i): (vx, vy, vz) for i, vx, vy, vz in zip(sim.species[1].id, sim.species[1].vx,
                                                        sim.species[1].vy, sim.species[1].vz)}
    sim.step()
    sp = sim.species[1]
    v = np.array([v0[int(i)] for i in sp.id])
    vp = np.stack([sp.vx, sp.vy, sp.vz], 1)
    hit = np.any(vp != v, axis=1)
    assert abs(hit.mean() - (1 - np.exp(-0.5))) < 5 * np.sqrt(0.4 * 0.6 / n)
    e_in = np.sum(v[hit] ** 2, 1)
    e_out = np.sum(vp[hit] ** 2, 1)
    recoil = (m_ion / m_n) * np.sum((v[hit] - vp[hit]) ** 2, 1)
    assert np.abs(e_in - e_out - recoil).max() <= 1e-12 * speed ** 2
    frac = e_out / e_in
    expect = (m_ion ** 2 + m_n ** 2) / (m_ion + m_n) ** 2
    assert abs(frac.mean() - expect) < 5 * frac.std() / np.sqrt(frac.size)


def _old_energy(sp, m):
    return 0.5 * m * (sp.vx ** 2 + sp.vy ** 2 + sp.vz ** 2) / W.QE


def test_ionization_pays_the_threshold_and_spawns_a_neutral_temperature_ion():
    """Every ionizing electron pays eps_th; the rest is shared between the parent and the new
    electron, so e_parent + e_new = eps - eps_th for every pair, with the parent's share
    uniform on [0, 1).  The pair is spawned at the parent's position with ids next_id + 2k
    (electron) and + 1 (ion), k the parent's rank in list order; the ion takes a velocity from
    the neutral Maxwellian: zero mean, variance T_gas qe / M_neutral per component.  Fails
    for: the energy split taken before paying the threshold, both shares drawn independently,
    pairs ranked in another order, or the ion's thermal speed from the ion or electron mass."""
    from scipy import stats
    n = 400_000
    eps = 60.0
    speed = np.sqrt(2 * eps * W.QE / W.ME)
    sig_el, sig0, th = 6e-20, 1e-20, 24.6
    ng, dt = 2e23, 2e-12
    t_gas, m_n = 0.3, 40 * W.AMU
    mesh = O.Mesh(4, 4, 0.25, 0, O.BC_PERIODIC, O.BC_PERIODIC)
    cfg = W.base_config(precision=W.FP64, n_species=2, dt=dt, eps0=1.0, q=[-W.QE, W.QE],
                        m=[W.ME, 4 * W.AMU], qe=W.QE, mcc=1, gas_density=ng, gas_temperature_ev=t_gas,
                        neutral_mass=m_n, sigma_el=sig_el, sigma_iz0=sig0, eps_th_ev=th)
    sim = O.Sim(cfg, mesh)
    rng = np.random.default_rng(2)
    x = rng.random(n); y = rng.random(n)
    d = rng.standard_normal((3, n)); d /= np.linalg.norm(d, axis=0)
    sim.load(0, x, y, speed * d[0], speed * d[1], speed * d[2], np.zeros(n))
    sim.load(1, x[:0], y[:0], x[:0], x[:0], x[:0], x[:0])
    old_ids = sim.species[0].id.copy()
    sim.step()
    e, ion = sim.species[0], sim.species[1]
    by_id = {int(i): k for k, i in enumerate(e.id)}
    ion_by_id = {int(i): k for k, i in enumerate(ion.id)}
    en = _old_energy(e, W.ME)
    rest = eps - th
    # parents: original electrons left with at most eps - eps_th (elastic ones keep ~eps)
    parents = [int(i) for i in old_ids if en[by_id[int(i)]] <= rest * (1 + 1e-12)]
    k = len(parents)
    assert k == ion.n and e.n == n + k and k > 2000
    e1 = np.array([en[by_id[p]] for p in parents])
    e2 = np.array([en[by_id[n + 2 * r]] for r in range(k)])
    assert np.abs(e1 + e2 - rest).max() <= 1e-12 * rest
    assert stats.kstest(e1 / rest, "uniform").pvalue > 1e-4
    for r, p in enumerate(parents):
        a, b, c = by_id[p], by_id[n + 2 * r], ion_by_id[n + 2 * r + 1]
        assert e.x[a] == e.x[b] == ion.x[c] and e.y[a] == e.y[b] == ion.y[c]
    vi = np.stack([ion.vx, ion.vy, ion.vz])
    var = t_gas * W.QE / m_n
    assert np.abs(vi.mean(axis=1)).max() < 5 * np.sqrt(var / k)
    s2 = (vi ** 2).mean()
    assert abs(s2 / var - 1) < 5 * np.sqrt(2.0 / (3 * k))
    # the new electrons' directions are isotropic
    be = np.array([by_id[n + 2 * r] for r in range(k)])
    dz = e.vz[be] / np.sqrt(2 * e2 * W.QE / W.ME)
    assert abs((dz ** 2).mean() - 1 / 3) < 5 * np.sqrt(4 / 45 / k)


# --------------------------------------------------------------------------------------
# Corner and centre fields (§3: E on cell nodes/corners; the adaptation's |E| criterion)
# --------------------------------------------------------------------------------------
def _disk_mesh(n, lmax, bcx, bcy):
    r, l, m = _disk_tree(n, lmax)
    return O.Mesh(n, n, 1.0 / n, lmax, bcx, bcy, r, l, m)


def test_cell_emag_exact_for_linear_potentials_on_amr():
    """|E| at leaf centres from the face gradients is exact for a linear potential on a
    four-level tree, at coarse-fine faces and at the walls (Dirichlet along the gradient,
    Neumann across it).  Fails for: a coarse-fine gradient taken over h instead of 3h/4, a
    wall gradient over h instead of h/2, or a dropped factor of one half in the averages."""
    n = 8
    a, b = 2.5, -1.75
    M = _disk_mesh(n, 3, O.BC_DIRICHLET, O.BC_NEUMANN)
    assert len(np.unique(M.s)) == 4
    xc, yc = M.centres()
    em = M.cell_emag(a * xc, [0.0, a * M.lx, 0.0, 0.0])
    assert np.abs(em - abs(a)).max() < 1e-12
    M = _disk_mesh(n, 3, O.BC_NEUMANN, O.BC_DIRICHLET)
    xc, yc = M.centres()
    em = M.cell_emag(b * yc, [0.0, 0.0, 0.0, b * M.ly])
    assert np.abs(em - abs(b)).max() < 1e-12
    # both components: leaves away from the walls
    M = _disk_mesh(n, 3, O.BC_DIRICHLET, O.BC_DIRICHLET)
    xc, yc = M.centres()
    em = M.cell_emag(a * xc + b * yc, [0.0, 0.0, 0.0, 0.0])
    inner = (M.ix > 0) & (M.iy > 0) & (M.ix + M.s < (n << 3)) & (M.iy + M.s < (n << 3))
    assert inner.sum() > 100
    assert np.abs(em[inner] - np.hypot(a, b)).max() < 1e-12


def test_node_e_on_a_uniform_mesh_is_the_compact_four_cell_formula():
    """On a uniform periodic mesh the corner field of any potential is the compact formula
    E_x = -[(phi_{i+1,j} - phi_{i,j}) + (phi_{i+1,j+1} - phi_{i,j+1})] / 2h (E_y likewise) of
    the four cells around the node, and it is exact at every node for a quadratic potential.
    Fails for: a face gradient taken on the wrong side of the node, one of the two incident
    faces dropped, or a corner index transposed."""
    n = 16
    h = 1.0 / n
    M = O.Mesh(n, n, h, 0, O.BC_PERIODIC, O.BC_PERIODIC)
    rng = np.random.default_rng(8)
    phi = rng.standard_normal(M.nleaf)
    E = M.node_e(phi, [0, 0, 0, 0])
    g = np.zeros((n, n)); g[M.iy, M.ix] = phi        # g[j, i]
    # node (I, J) at the lower-left corner of cell (I, J): cells I-1, I and J-1, J around it
    gl, gd, gld = np.roll(g, 1, axis=1), np.roll(g, 1, axis=0), np.roll(np.roll(g, 1, axis=0), 1, axis=1)
    ex = -((g - gl) + (gd - gld)) / (2 * h)
    ey = -((g - gd) + (gl - gld)) / (2 * h)
    for c, (di, dj) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
        I = (M.ix + di) % n; J = (M.iy + dj) % n
        assert np.abs(E[:, c, 0] - ex[J, I]).max() < 1e-12 * n
        assert np.abs(E[:, c, 1] - ey[J, I]).max() < 1e-12 * n
    # quadratic potential on a Dirichlet box: exact at interior nodes
    M = O.Mesh(n, n, h, 0, O.BC_DIRICHLET, O.BC_DIRICHLET)
    xc, yc = M.centres()
    phi = 0.7 * xc ** 2 - 1.3 * xc * yc + 0.4 * yc ** 2 + 0.2 * xc
    E = M.node_e(phi, [0, 0, 0, 0])
    for c, (di, dj) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
        X = (M.ix + di) * h; Y = (M.iy + dj) * h
        inner = (X > 0) & (X < 1) & (Y > 0) & (Y < 1)
        ex = -(1.4 * X - 1.3 * Y + 0.2); ey = -(-1.3 * X + 0.8 * Y)
        assert np.abs(E[inner, c, 0] - ex[inner]).max() < 1e-12
        assert np.abs(E[inner, c, 1] - ey[inner]).max() < 1e-12


@pytest.mark.parametrize("seed,px,py", [(4, True, True), (5, False, True)])
def test_node_e_is_continuous_across_hanging_nodes(seed, px, py):
    """On a 2:1 tree, a corner of a fine leaf that lies inside the edge of a coarser leaf must
    carry the value of the coarse leaf's bilinear field there (the mean of that edge's two
    corner values), for any potential, so that the gathered field is continuous.  Fails for:
    a hanging node treated as a regular node, or the mean taken over the ends of another edge."""
    nx0, ny0, lmax = 4, 3, 3
    r, l, m = W.random_tree(nx0, ny0, lmax, 0.35, seed, px, py)
    M = O.Mesh(nx0, ny0, 0.25, lmax, O.BC_PERIODIC if px else O.BC_DIRICHLET,
               O.BC_PERIODIC if py else O.BC_NEUMANN, r, l, m)
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal(M.nleaf)
    E = M.node_e(phi, [0.3, -0.2, 0.0, 0.0])
    NX, NY = nx0 << lmax, ny0 << lmax
    checked = 0
    for A in range(M.nleaf):
        for c, (di, dj) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
            I, J = M.ix[A] + di * M.s[A], M.iy[A] + dj * M.s[A]
            # leaves on the four lattice cells around the node
            around = [M.leaf_at(I - 1, J - 1), M.leaf_at(I, J - 1), M.leaf_at(I - 1, J), M.leaf_at(I, J)]
            for B in set(around) - {-1, A}:
                if M.s[B] != 2 * M.s[A]:
                    continue
                # node strictly inside an edge of B (periodic distances on the lattice)
                oi = (I - M.ix[B]) % NX if px else I - M.ix[B]
                oj = (J - M.iy[B]) % NY if py else J - M.iy[B]
                sB = M.s[B]
                if oi in (0, sB) and 0 < oj < sB:      # vertical edge of B: corners below/above
                    k0, k1 = (0, 2) if oi == 0 else (1, 3)
                elif oj in (0, sB) and 0 < oi < sB:    # horizontal edge
                    k0, k1 = (0, 1) if oj == 0 else (2, 3)
                else:
                    continue
                ref = 0.5 * (E[B, k0] + E[B, k1])
                assert np.abs(E[A, c] - ref).max() <= 1e-12 * np.abs(E).max(), (A, c, B)
                checked += 1
    assert checked > 20


def test_node_e_and_cell_emag_converge_for_a_smooth_potential_on_amr():
    """For phi = sin(pi x) sin(pi y) sampled at the leaf centres of a three-level tree (walls at
    phi = 0), the corner field converges to -grad phi at the corners and |E| to |grad phi| at
    the centres as the mesh is refined: observed order >= 0.95 in the max norm (first order at
    hanging nodes and walls) and >= 1.3 in the mean square.  Fails for: a dropped term of
    the corner average or of the wall gradient, a sign error, or E taken at the leaf centre."""
    errs = []
    for n in (16, 32, 64):
        M = _disk_mesh(n, 2, O.BC_DIRICHLET, O.BC_DIRICHLET)
        xc, yc = M.centres()
        phi = np.sin(np.pi * xc) * np.sin(np.pi * yc)
        E = M.node_e(phi, [0, 0, 0, 0])
        h = M.h()
        X = (M.ix * M.hf)[:, None] + np.array([0, 1, 0, 1])[None, :] * h[:, None]
        Y = (M.iy * M.hf)[:, None] + np.array([0, 0, 1, 1])[None, :] * h[:, None]
        ex = -np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
        ey = -np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
        en = np.maximum(np.abs(E[:, :, 0] - ex), np.abs(E[:, :, 1] - ey))
        em = M.cell_emag(phi, [0, 0, 0, 0])
        ec = np.abs(em - np.pi * np.hypot(np.cos(np.pi * xc) * np.sin(np.pi * yc),
                                          np.sin(np.pi * xc) * np.cos(np.pi * yc)))
        errs.append((en.max(), np.sqrt((en ** 2).mean()), ec.max(), np.sqrt((ec ** 2).mean())))
    e = np.array(errs)
    order = np.log2(e[:-1] / e[1:])
    assert order[:, 0].min() >= 0.95 and order[:, 2].min() >= 0.95, order
    assert order[:, 1].min() >= 1.3 and order[:, 3].min() >= 1.3, order


# --------------------------------------------------------------------------------------
# Time averages (§3.3 RF-cycle averages of n_e, n_i, T_e, phi and the EEDF; §3.1 reset)
# --------------------------------------------------------------------------------------
def _static_sim(n, te_ev, seed=3, n_bins=64, eps_max=40.0):
    """Electrons and ions that do not move (zero time step) on a uniform Dirichlet mesh with a
    fixed wall potential: every step samples the same state."""
    cfg = W.base_config(precision=W.FP64, n_species=2, dt=1e-30, eps0=W.EPS0, q=[-W.QE, W.QE],
                        m=[W.ME, 4 * W.AMU], qe=W.QE, bc_x=W.BC_DIRICHLET, bc_y=W.BC_NEUMANN,
                        phi_right=5.0)
    M = O.Mesh(8, 4, 0.25, 0, O.BC_DIRICHLET, O.BC_NEUMANN)
    sim = O.Sim(cfg, M)
    rng = np.random.default_rng(seed)
    vt = np.sqrt(te_ev * W.QE / W.ME)
    for s in (0, 1):
        x = rng.random(n) * M.lx; y = rng.random(n) * M.ly
        v = rng.standard_normal((3, n)) * (vt if s == 0 else 0.0)
        sim.load(s, x, y, v[0], v[1], v[2], rng.random(n) + 0.5)
    sim.diag_enable(n_bins, eps_max)
    return sim


def test_time_averages_of_a_static_state_equal_the_state():
    """A state that does not change (zero time step): the averages over 5 steps equal the
    instantaneous densities per leaf, the potential of the solve, and T_e = (2/3) <eps> of each
    leaf's electrons; counts in the energy histogram are exact (5 x the weights per bin).
    Fails for: a missing division by the sample count or by the leaf area, the 2/3, or a
    sample taken twice per step."""
    sim = _static_sim(4000, 2.0)
    sim.step(5)
    d = sim.diag_fields()
    e, i = sim.species
    area = sim.mesh.area()
    ne = np.bincount(e.leaf, weights=e.w, minlength=sim.mesh.nleaf) / area
    ni = np.bincount(i.leaf, weights=i.w, minlength=sim.mesh.nleaf) / area
    eps = 0.5 * W.ME * (e.vx ** 2 + e.vy ** 2 + e.vz ** 2) / W.QE
    te = (2.0 / 3.0) * np.bincount(e.leaf, weights=e.w * eps, minlength=sim.mesh.nleaf) / (ne * area)
    assert np.allclose(d["ne"], ne, rtol=1e-13) and np.allclose(d["ni"], ni, rtol=1e-13)
    assert np.allclose(d["te"], te, rtol=1e-13)
    assert np.allclose(d["phi"], sim.phi, rtol=1e-13, atol=1e-13)
    f, k = sim.diag_eedf()
    assert k == 5
    counts = np.bincount(np.floor(eps / (40.0 / 64)).astype(int)[eps < 40.0],
                         weights=e.w[eps < 40.0], minlength=64)
    assert np.allclose(f * 5 * counts.sum() * (40.0 / 64), 5 * counts, rtol=1e-12)


def test_eedf_of_a_maxwellian_is_the_maxwell_distribution_and_te_its_temperature():
    """Electrons from a Maxwellian at T (isotropic, no drift): the EEDF is
    f(eps) = 2 sqrt(eps / pi) T^(-3/2) exp(-eps / T) per eV (chi-square over bins with >= 20
    expected counts) and the averaged T_e = (2/3) <eps> = T within sampling error.  Fails
    for: a histogram of speeds instead of energies, a missing factor 1/2 in eps, bins off by
    one."""
    from scipy import stats
    T = 3.0
    sim = _static_sim(40000, T, n_bins=40, eps_max=20.0)
    e = sim.species[0]
    e.w[:] = 1.0   # equal weights: the histogram is a plain count
    sim.step(1)
    f, k = sim.diag_eedf()
    edges = np.linspace(0.0, 20.0, 41)
    cdf = stats.gamma(1.5, scale=T).cdf(edges)       # eps / T ~ Gamma(3/2) for a 3D Maxwellian
    p = np.diff(cdf) / (cdf[-1] - cdf[0])
    n_in = int(np.count_nonzero(0.5 * W.ME * (e.vx ** 2 + e.vy ** 2 + e.vz ** 2) / W.QE < 20.0))
    obs = f * (20.0 / 40) * n_in
    exp = p * n_in
    ok = exp >= 20
    chi2 = np.sum((obs[ok] - exp[ok]) ** 2 / exp[ok])
    assert stats.chi2(ok.sum() - 1).sf(chi2) > 1e-4
    d = sim.diag_fields()
    te_all = (2.0 / 3.0) * np.sum(e.w * 0.5 * W.ME * (e.vx ** 2 + e.vy ** 2 + e.vz ** 2) / W.QE) / e.w.sum()
    assert abs(te_all / T - 1) < 5 * np.sqrt(2.0 / (3 * e.n))
    assert np.all(d["te"][d["ne"] > 0] > 0)


def test_time_averages_restart_when_the_grid_changes():
    """§3.1: statistics counters are reset when the grid changes; an adaptation that changes
    no leaf keeps them."""
    sim = _static_sim(2000, 2.0)
    sim.cfg.update(max_level=1, refine_count=10 ** 9, coarsen_count=-1, e_ref=1e30)
    sim.step(3)
    sim.adapt(mesh=True, particles=False)
    assert sim.diag["samples"] == 3
    sim.cfg.update(refine_count=10)
    M = O.Mesh(8, 4, 0.25, 1, O.BC_DIRICHLET, O.BC_NEUMANN)
    sim2 = O.Sim(dict(sim.cfg), M)
    for s in (0, 1):
        sp = sim.species[s]
        sim2.load(s, sp.x, sp.y, sp.vx, sp.vy, sp.vz, sp.w)
    sim2.diag_enable(64, 40.0)
    sim2.step(3)
    st = sim2.adapt(mesh=True, particles=False)["mesh"]
    assert st["refined"] > 0 and sim2.diag["samples"] == 0 and sim2.diag["we"].size == sim2.mesh.nleaf


# --------------------------------------------------------------------------------------
# Cloud-in-cell shapes on uniform meshes (§3: CIC-EM momentum-conserving, CIC-EC energy-
# conserving)
# --------------------------------------------------------------------------------------
def _cic_weights_of(x, y, nx, ny, h, px=True, py=True):
    """The charge each cell receives from a unit charge at (x, y), from the oracle's deposit."""
    Q = np.zeros(nx * ny)
    O.lib().or_cic_deposit(nx, ny, h, int(px), int(py), 1, O._ptr(np.array([x])), O._ptr(np.array([y])),
                           O._ptr(np.array([1.0])), 1.0, O._ptr(Q))
    return Q


def test_cic_weights_are_the_overlap_of_a_cell_sized_cloud():
    """The CIC weight of a cell is the area of the cell shared with a square of the cell's size
    centred on the particle (worked out geometrically here), in the interior; a particle at a
    cell centre gives that cell everything; at a Dirichlet wall the weight beyond the wall folds
    into the boundary cell, so the total stays 1.  Fails for: weights of the wrong corner,
    a half-cell offset missing, or the folded weight dropped."""
    nx, ny, h = 8, 6, 0.5
    rng = np.random.default_rng(3)
    for _ in range(50):
        x, y = 1.0 + 2.0 * rng.random(), 1.0 + 1.0 * rng.random()
        Q = _cic_weights_of(x, y, nx, ny, h)
        ref = np.zeros(nx * ny)
        for j in range(ny):
            for i in range(nx):
                ox = max(0.0, min(x + h / 2, (i + 1) * h) - max(x - h / 2, i * h))
                oy = max(0.0, min(y + h / 2, (j + 1) * h) - max(y - h / 2, j * h))
                ref[i + nx * j] = ox * oy / (h * h)
        assert np.abs(Q - ref).max() < 1e-14
    Q = _cic_weights_of(2.75, 1.25, nx, ny, h)
    assert Q[5 + nx * 2] == 1.0 and Q.sum() == 1.0
    Q = _cic_weights_of(0.1, 1.25, nx, ny, h, px=False)       # within half a cell of x = 0
    assert abs(Q.sum() - 1.0) < 1e-15 and Q[0 + nx * 2] == 1.0


def _cic_sim(shape, n=60, seed=4, bcx=W.BC_PERIODIC):
    M = O.Mesh(16, 8, 0.125, 0, bcx, O.BC_PERIODIC)
    cfg = W.base_config(precision=W.FP64, n_species=1, dt=0.01, eps0=1.0, q=[-1.0], m=[1.0], bc_x=bcx,
                        bc_y=W.BC_PERIODIC, shape=shape, phi_right=0.7)
    sim = O.Sim(cfg, M)
    rng = np.random.default_rng(seed)
    x = rng.random(n) * M.lx; y = rng.random(n) * M.ly; w = rng.random(n) + 0.5
    z = np.zeros(n)
    cfg["rho_background"] = w.sum() / (M.lx * M.ly)             # neutral periodic box
    sim.load(0, x, y, z, z, z, w)
    sim.fields()
    return sim


def test_cic_em_conserves_momentum_and_cic_ec_does_not():
    """CIC-EM gathers E (central differences at the cell centres) with the deposit's weights,
    so the total force on all particles of a periodic box vanishes to rounding (no self-force,
    action equals reaction); CIC-EC's gradient of the interpolated potential does not.  Fails
    for: an EM gather whose weights differ from the deposit's (e.g. the nearest centre), or
    one-sided differences."""
    for shape, zero in ((1, True), (2, False)):
        sim = _cic_sim(shape)
        sp = sim.species[0]
        ex, ey = sim.cic_field(sp)
        F = np.array([np.sum(sp.q * sp.w * ex), np.sum(sp.q * sp.w * ey)])
        scale = np.sum(np.abs(sp.q * sp.w) * np.hypot(ex, ey))
        assert (np.abs(F).max() < 1e-12 * scale) == zero, (shape, F, scale)


def test_cic_ec_force_is_minus_the_gradient_of_the_interpolated_potential():
    """CIC-EC: E at a particle is -grad of Phi(x) = sum_c W_c(x) phi_c with the deposit's own
    weights W_c (taken here from the deposit of a unit charge), checked by central differences
    inside one cell quarter (Phi is bilinear there, so they are exact); CIC-EM is not.  Fails
    for: EM-style gathering of centre fields, or a sign error."""
    for shape in (1, 2):
        sim = _cic_sim(shape)
        M = sim.mesh
        rng = np.random.default_rng(9)
        worst = 0.0
        for _ in range(40):
            # a point in the interior of a cell quarter, at least d away from its edges
            i, j = rng.integers(0, 2 * M.nx0), rng.integers(0, 2 * M.ny0)
            q = M.h0 / 2
            x, y = (i + 0.2 + 0.6 * rng.random()) * q, (j + 0.2 + 0.6 * rng.random()) * q
            d = 0.05 * q
            phi_at = lambda a, b: _cic_weights_of(a, b, M.nx0, M.ny0, M.h0) @ sim.phi
            gx = (phi_at(x + d, y) - phi_at(x - d, y)) / (2 * d)
            gy = (phi_at(x, y + d) - phi_at(x, y - d)) / (2 * d)
            sp = O.Species(-1.0, 1.0, np.array([x]), np.array([y]), *[np.zeros(1) for _ in range(4)],
                           np.zeros(1, np.uint64), M.locate([x], [y]))
            ex, ey = sim.cic_field(sp)
            worst = max(worst, abs(ex[0] + gx), abs(ey[0] + gy))
        scale = np.abs(np.diff(sim.phi)).max() / M.h0
        assert (worst < 1e-9 * scale) == (shape == 2), (shape, worst, scale)


@pytest.mark.parametrize("shape", [1, 2])
def test_cic_uniform_field_between_plates_is_exact(shape):
    """No charge, plates at x = 0 (0 V) and x = Lx (0.7 V): phi is linear and both gathers give
    E = -0.7 / Lx at every particle, walls included."""
    M = O.Mesh(16, 8, 0.125, 0, O.BC_DIRICHLET, O.BC_PERIODIC)
    cfg = W.base_config(precision=W.FP64, n_species=1, dt=0.01, eps0=1.0, q=[-1.0], m=[1.0],
                        bc_x=W.BC_DIRICHLET, bc_y=W.BC_PERIODIC, shape=shape, phi_right=0.7)
    sim = O.Sim(cfg, M)
    rng = np.random.default_rng(2)
    n = 200
    x = rng.random(n) * M.lx; y = rng.random(n) * M.ly; z = np.zeros(n)
    sim.load(0, x, y, z, z, z, z)
    sim.fields()
    ex, ey = sim.cic_field(sim.species[0])
    assert np.abs(ex + 0.7 / M.lx).max() < 1e-12 and np.abs(ey).max() < 1e-12


def test_cic_deposit_conserves_charge_at_walls():
    sim = _cic_sim(1, bcx=W.BC_DIRICHLET)
    sp = sim.species[0]
    Q = sim.charge()
    assert abs(Q.sum() - sp.q * sp.w.sum()) < 1e-13 * sp.w.sum()
