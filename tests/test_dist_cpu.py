"""The multi-rank path of the benchmark on the CPU (gloo, two ranks): the whole-job
aggregation (slowest rank's time, particle-steps of all ranks) and the reference arm under
torchrun (rank 0 alone runs and prints, the other rank exits without work)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank = dist.get_rank()
t, ps = bench._aggregate(1.0 + rank, 100 * (rank + 1), dist.get_world_size(), "cpu")
print(json.dumps({{"rank": rank, "t": t, "ps": ps}}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = sorted((json.loads([l for l in o.splitlines() if l.startswith("{")][-1]) for o, _ in outs),
                 key=lambda d: d["rank"])
    for d in res:
        assert d["t"] == 2.0 and d["ps"] == 300.0  # max of 1 and 2 seconds; 100 + 200 particle-steps


def test_aggregate_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._aggregate(1.5, 42, 1, "cpu") == (1.5, 42.0)


def test_reference_arm_under_torchrun_two_ranks():
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl",
                        "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


SHARD_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch, torch.distributed as dist
dist.init_process_group("gloo")
from paper_1604_07713_gb300 import workloads as W
from paper_1604_07713_gb300.shard import lpt_shard
rank, ws = dist.get_rank(), dist.get_world_size()
members = W.ensemble(256)
costs = [m[3] for m in members]
mine = lpt_shard(costs, ws)[rank]
# every rank sees the whole assignment only through the aggregation of its own share
n = torch.tensor([len(mine), sum(costs[i] for i in mine)], dtype=torch.float64)
tot = n.clone(); dist.all_reduce(tot)
mx = n.clone(); dist.all_reduce(mx, op=dist.ReduceOp.MAX)
print(json.dumps({{"rank": rank, "mine": mine, "total": tot.tolist(), "max": mx.tolist()}}))
dist.destroy_process_group()
"""


def test_ensemble_instances_split_over_two_gloo_ranks_by_lpt():
    """§8(e): the ensemble's independent instances split over the ranks with no exchange; the
    two ranks' shares are disjoint, cover all 256 instances and balance the particle counts
    within Graham's LPT bound."""
    sys.path.insert(0, ROOT)
    from paper_1604_07713_gb300 import workloads as W
    costs = [m[3] for m in W.ensemble(256)]
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", SHARD_WORKER.format(root=ROOT)], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = sorted((json.loads([l for l in o.splitlines() if l.startswith("{")][-1]) for o, _ in outs),
                 key=lambda d: d["rank"])
    a, b = set(res[0]["mine"]), set(res[1]["mine"])
    assert not (a & b) and a | b == set(range(256))
    assert res[0]["total"] == [256.0, float(sum(costs))]
    bound = (4.0 / 3.0 - 1.0 / 6.0) * max(sum(costs) / 2.0, max(costs))
    assert res[0]["max"][1] <= bound
    # LPT on this list is far tighter than the bound in practice
    assert res[0]["max"][1] <= 1.01 * sum(costs) / 2.0


def test_lpt_shard_hand_case():
    sys.path.insert(0, ROOT)
    from paper_1604_07713_gb300.shard import lpt_shard
    # costs 7, 6, 5, 4, 3, 2 on 2 ranks (loads after each): 7 -> 0 (7, 0); 6 -> 1 (7, 6);
    # 5 -> 1 (7, 11); 4 -> 0 (11, 11); 3 -> 0 on the tie (14, 11); 2 -> 1 (14, 13)
    assert lpt_shard([7, 6, 5, 4, 3, 2], 2) == [[0, 3, 4], [1, 2, 5]]
    assert lpt_shard([1, 1, 1], 1) == [[0, 1, 2]]
    assert lpt_shard([5], 3) == [[0], [], []]
