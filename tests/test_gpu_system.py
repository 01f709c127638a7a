"""System behaviour of the C ABI on the GPU: batched instances equal the same instances run
alone, runs are deterministic, capacity grows under ionization, and invalid input is
refused with the documented status."""
import numpy as np
import pytest

import paper_1604_07713_gb300 as G
from paper_1604_07713_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    G.build()


def _ccp(nx, ppc, seed, volt, ng):
    cfg, mesh, parts = W.ccp(nx=nx, ny=8, ppc=ppc, seed=seed, precision=W.FP32, volt=volt, ng=ng, te=8.0)
    return cfg, mesh, parts


def _run_alone(cfg, mesh, parts, steps):
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        for s in sorted(parts):
            ctx.load(s, **parts[s])
        ctx.step(steps)
        return [ctx.particles(s) for s in (0, 1)]


def test_batched_instances_equal_instances_run_alone():
    cases = [_ccp(32, 10, 1, 100.0, 3e20), _ccp(48, 20, 2, 300.0, 1e21), _ccp(64, 15, 3, 200.0, 3e21)]
    for i, (cfg, _, _) in enumerate(cases):
        cfg["instance"] = i
    with G.Context([c[0] for c in cases]) as ctx:
        for i, (cfg, mesh, parts) in enumerate(cases):
            ctx.set_mesh_dict(mesh, inst=i)
            for s in sorted(parts):
                ctx.load(s, **parts[s], inst=i)
        ctx.step(4)
        batched = [[ctx.particles(s, inst=i) for s in (0, 1)] for i in range(len(cases))]
    for i, (cfg, mesh, parts) in enumerate(cases):
        alone = _run_alone(cfg, mesh, parts, 4)
        for s in (0, 1):
            for k in ("id", "x", "y", "vx", "vy", "vz", "w"):
                assert np.array_equal(batched[i][s][k], alone[s][k]), (i, s, k)


def test_two_runs_are_bitwise_identical():
    cfg, mesh, parts = _ccp(64, 20, 5, 200.0, 3e21)
    a = _run_alone(cfg, mesh, parts, 5)
    b = _run_alone(cfg, mesh, parts, 5)
    for s in (0, 1):
        for k in a[s]:
            assert np.array_equal(a[s][k], b[s][k])


def test_capacity_grows_under_ionization_and_fixed_capacity_is_enforced():
    cfg, mesh, parts = W.ccp(nx=32, ny=8, ppc=20, seed=9, precision=W.FP32, te=40.0, ng=3e21)
    cfg["dt"] *= 4
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        for s in sorted(parts):
            ctx.load(s, **parts[s])
        n0 = ctx.counts()
        ctx.step(6)
        n1 = ctx.counts()
        assert n1["n_i"] > n0["n_i"]  # ionization spawned pairs
        ids = ctx.particles(0)["id"]
        assert np.unique(ids).size == ids.size
    cfg["particle_capacity"] = parts[0]["x"].size + 1
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        for s in sorted(parts):
            ctx.load(s, **parts[s])
        with pytest.raises(G.PicError) as e:
            ctx.step(6)
        assert e.value.status == G.PIC_ECAPACITY


def test_invalid_input_is_refused():
    cfg, mesh, parts = _ccp(16, 4, 1, 100.0, 1e20)
    with G.Context(cfg) as ctx:
        ctx.set_mesh_dict(mesh)
        p = {k: v.copy() for k, v in parts[0].items()}
        p["x"][3] = -1.0  # outside the domain
        with pytest.raises(G.PicError) as e:
            ctx.load(0, **p)
        assert e.value.status == G.PIC_EINVAL and "outside" in str(e.value)
    # a leaf set that is not 2:1 balanced across faces
    cfg2 = W.base_config(precision=W.FP32, n_species=1, q=[-1.0], m=[1.0], bc_x=W.BC_DIRICHLET,
                         bc_y=W.BC_NEUMANN, max_level=2)
    root, level, morton = [0] * 16 + [1], [2] * 16 + [0], list(range(16)) + [0]
    with G.Context(cfg2) as ctx:
        with pytest.raises(G.PicError) as e:
            ctx.set_mesh(0, 2, 1, 1.0, np.array(root), np.array(morton), np.array(level))
        assert e.value.status == G.PIC_EINVAL


def test_ensemble_steps_replay_one_graph_and_match_uncaptured_steps():
    # from the second step on, the steps of an ensemble in steady state are one graph replay;
    # the result is the same, bit for bit, as stepping without the graph (one instance alone)
    cases = [_ccp(32, 10, 4, 150.0, 1e21), _ccp(40, 12, 5, 250.0, 2e21)]
    for i, (cfg, _, _) in enumerate(cases):
        cfg["instance"] = i
    with G.Context([c[0] for c in cases]) as ctx:
        for i, (cfg, mesh, parts) in enumerate(cases):
            ctx.set_mesh_dict(mesh, inst=i)
            for s in sorted(parts):
                ctx.load(s, **parts[s], inst=i)
        ctx.step(1)
        G.pic_set_timing(ctx.ctx, True)
        for _ in range(3):
            ctx.step(1)
        ph = G.pic_get_timing(ctx.ctx)
        G.pic_set_timing(ctx.ctx, False)
        # replays, their phases timed inside the graph: two batched pushes per replay
        assert ph["graph"][1] > 0 and ph["move"][1] == 3 * 2
        assert 0.0 < sum(v[0] for k, v in ph.items() if k != "graph") <= ph["graph"][0] * 1.01 + 0.05
        batched = [[ctx.particles(s, inst=i) for s in (0, 1)] for i in range(len(cases))]
    for i, (cfg, mesh, parts) in enumerate(cases):
        alone = _run_alone(cfg, mesh, parts, 4)
        for s in (0, 1):
            for k in ("id", "x", "vx", "w"):
                assert np.array_equal(batched[i][s][k], alone[s][k]), (i, s, k)


def test_batched_step_is_one_launch_per_phase_and_repairs_like_alone():
    """The captured ensemble step runs every instance's phases in one launch each (about 20
    graph nodes per step, whatever the number of instances), and its list repairs (tail moves,
    re-layouts, spawned ions overflowing) equal those of each instance stepping alone."""
    from test_gpu_lists import _beam_case
    beam_iz = _beam_case(W.FP64, ionize=True)
    tight = _beam_case(W.FP64, ionize=False, seed=12)
    tight[0]["particle_capacity"] = tight[2][0]["x"].size + 40  # little room at the tail
    cases = [beam_iz, tight, W.ccp(nx=32, ny=8, ppc=10, seed=3, precision=W.FP64, volt=200.0, ng=1e21, te=8.0)]
    for i, (cfg, _, _) in enumerate(cases):
        cfg["instance"] = i
    steps = 4
    with G.Context([c[0] for c in cases]) as ctx:
        for i, (cfg, mesh, parts) in enumerate(cases):
            ctx.set_mesh_dict(mesh, inst=i)
            for s in sorted(parts):
                ctx.load(s, **parts[s], inst=i)
        ctx.step(1)
        before = [[G.pic_get_list_stats(ctx.ctx, i, s) for s in (0, 1)] for i in range(len(cases))]
        G.pic_set_timing(ctx.ctx, True)
        ctx.step(steps - 1)
        ph = G.pic_get_timing(ctx.ctx)
        G.pic_set_timing(ctx.ctx, False)
        after = [[G.pic_get_list_stats(ctx.ctx, i, s) for s in (0, 1)] for i in range(len(cases))]
        batched = [[ctx.particles(s, inst=i) for s in (0, 1)] for i in range(len(cases))]
    assert ph["move"][1] == 2 * (steps - 1) and ph["graph"][1] > 0  # every later step was a replay
    assert ph["graph"][1] <= 24 * (steps - 1), ph["graph"]  # launches per replay
    # the replays repaired lists: tail moves of the beam's electrons and spawned ions; the
    # tight instance's electrons were laid out again (and repaired during the replays)
    assert after[0][0][1] > before[0][0][1] and after[0][1][1] > before[0][1][1]
    assert after[1][0][0] >= 1 and sum(after[1][0][:2]) > sum(before[1][0][:2])
    for i, (cfg, mesh, parts) in enumerate(cases):
        alone = _run_alone(cfg, mesh, parts, steps)
        for s in (0, 1):
            for k in ("id", "x", "y", "vx", "vy", "vz", "w"):
                assert np.array_equal(batched[i][s][k], alone[s][k]), (i, s, k)


@pytest.mark.parametrize("n_inst", [1, 3])
def test_autotuned_steps_equal_default_steps(n_inst):
    # the tuner's steps are ordinary steps under other launch shapes (push block size, blocks
    # per SM, the GPU share and branches of a captured ensemble step): the state after them
    # equals stepping with the default shapes, bit for bit
    cases = [_ccp(32 + 8 * i, 10, 4 + i, 150.0 + 50 * i, 1e21) for i in range(n_inst)]
    for i, (cfg, _, _) in enumerate(cases):
        cfg["instance"] = i

    def run(tune):
        with G.Context([c[0] for c in cases]) as ctx:
            for i, (cfg, mesh, parts) in enumerate(cases):
                ctx.set_mesh_dict(mesh, inst=i)
                for s in sorted(parts):
                    ctx.load(s, **parts[s], inst=i)
            used = ctx.autotune(11) if tune else 0
            ctx.step(12 - used)
            out = [[ctx.particles(s, inst=i) for s in (0, 1)] for i in range(n_inst)]
            return out, used, ctx.tuning()

    a, used, t = run(True)
    b, _, t0 = run(False)
    assert 5 <= used <= 11 and t["best_step_ms"] > 0.0 and t0["best_step_ms"] == 0.0
    assert t["push_threads"] in (128, 256) and t["graph_branches"] in (8, 16, 32)
    for i in range(n_inst):
        for s in (0, 1):
            for k in ("id", "x", "y", "vx", "vy", "vz", "w"):
                assert np.array_equal(a[i][s][k], b[i][s][k]), (i, s, k)
