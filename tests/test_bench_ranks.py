"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun would
launch them.  Every rank runs its own chain (replicas); the job's time is the
slowest rank's and its work the sum over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, work = bench.reduce_max_sum(1.5 + rank, 10.0 * (rank + 1), dist, "cpu")
    q.put((rank, t, work, bench.chain_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_the_summed_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]
    assert [o[2] for o in out] == [30.0, 30.0]
    assert out[0][3] != out[1][3]   # independent replicas


def test_single_rank_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_sum(3.0, 7.0) == (3.0, 7.0)


def test_cpu_legs_run_every_move_of_the_replay_workload():
    """The oracle leg of bench.py (cpu_baseline, and the reference arm) on the
    replay workload with joint pair moves and latent arrival times: it runs
    and counts every proposal type."""
    sys.path.insert(0, ROOT)
    import bench
    world, desc = bench._workload("replay", "variance", 0.1, 2.0, 0.2)
    assert "p_pair=0.1" in desc and "sig_a=2" in desc
    assert world.offsets is not None and (world.offsets != 0).any()
    base = bench._cpu_baseline(world, seconds_target=0.3, p_pair=0.1, sig_a=2.0, p_arr=0.2)
    assert base["kind"] == "oracle" and base["value"] > 0 and base["sweeps"] >= 1
    assert base["serial"]["cores"] == 1 and base["serial"]["value"] > 0 and base["serial"]["steps"] >= 1000
    st = {"proposed": [5, 6, 7], "pair": [2, 1, 0], "arrival": [3, 3, 1]}
    assert bench.n_proposals(st) == 23


def _shard_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import worldgen
    sizes = worldgen.batched_instances(256, seed=2000)
    costs = [bench.instance_cost(S, p) for S, p in sizes]
    mine = bench.shard_instances(costs, world, rank)
    gathered = bench.gather_summaries({"rank": rank, "instances": mine, "cost": sum(costs[i] for i in mine)}, dist)
    t, work = bench.reduce_max_sum(1.0 + rank, float(len(mine)), dist, "cpu")
    q.put((rank, mine, gathered, t, work))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_batched_instances():
    """The batched workload on two ranks: each rank computes its share of the
    256 instances from the same cost estimates, with no communication; the
    shares are disjoint, cover every instance and carry near-equal estimated
    cost; the summaries gathered after the timed region are the same on both
    ranks; time is the slowest rank's, work the sum."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = out[0][1], out[1][1]
    assert not set(a) & set(b) and sorted(a + b) == list(range(256))
    assert out[0][2] == out[1][2] and [g["rank"] for g in out[0][2]] == [0, 1]
    c0, c1 = out[0][2][0]["cost"], out[0][2][1]["cost"]
    assert abs(c0 - c1) <= 0.02 * (c0 + c1)
    assert [o[3] for o in out] == [2.0, 2.0] and [o[4] for o in out] == [256.0, 256.0]


@pytest.mark.parametrize("n", [1, 3, 8])
def test_instance_split_covers_and_balances(n):
    sys.path.insert(0, ROOT)
    import bench
    import worldgen
    costs = [bench.instance_cost(S, p) for S, p in worldgen.batched_instances(256, seed=2000)]
    shares = [bench.shard_instances(costs, n, r) for r in range(n)]
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(256))
    loads = [sum(costs[i] for i in s) for s in shares]
    # largest-first greedy: no share exceeds another by more than one instance
    assert max(loads) - min(loads) <= max(costs)


def test_instance_capacities_cover_the_density():
    """The capacities bench.py gives a batched instance: at least the
    defaults, growing with the events per region and the arrivals per
    station, capped at 512 events per region."""
    sys.path.insert(0, ROOT)
    import bench
    import worldgen
    sizes = worldgen.batched_instances(256, seed=2000)
    caps = [bench.instance_capacities(p) for _, p in sizes]
    assert all(ev >= 128 and fz >= 64 for ev, fz in caps)
    assert all(ev <= 512 for ev, _ in caps)
    dense = worldgen.ModelParams(W=300.0, T=900.0, Lambda=400.0)
    ev, fz = bench.instance_capacities(dense)
    per_region = dense.Lambda * dense.L ** 2 / dense.W ** 2
    assert ev >= per_region + bench.K_PER_PHASE and fz > 64
