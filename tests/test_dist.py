"""The benchmark's rank logic with two gloo ranks on the CPU: the split of
the scan's instances into disjoint, cost-balanced subsets (one per rank),
the barrier, the max over ranks of the per-rank times and the whole-job
throughput (no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2609_03550_b300 import inputs as I
    from paper_2609_03550_b300.ranks import Ranks, job_throughput, shard
    r = Ranks(backend="gloo")
    costs = [w.cell_modes() for w in I.batched_scan()]
    mine = shard(costs, r.world)[r.rank]
    r.barrier()
    t = 1.0 + rank  # rank 1 is the slowest
    tmax = r.max(t)
    value = job_throughput(sum(costs), tmax)
    r.barrier()
    q.put((rank, r.world, tmax, value, mine, sum(costs[i] for i in mine), sum(costs)))
    r.close()


def test_two_gloo_ranks_share_the_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    total = out[0][6]
    for _, w, tmax, value, _, _, _ in out:
        assert w == 2 and tmax == 2.0
        assert value == pytest.approx(total / 2.0)
    # the two subsets partition the 512 instances and carry nearly equal work
    a, b = out[0][4], out[1][4]
    assert sorted(a + b) == list(range(512)) and not set(a) & set(b)
    loads = [out[0][5], out[1][5]]
    assert loads[0] + loads[1] == total
    assert max(loads) / (total / 2) < 1.01


@pytest.mark.parametrize("world", [1, 3, 4, 8])
def test_shards_partition_and_balance(world):
    from paper_2609_03550_b300 import inputs as I
    from paper_2609_03550_b300.ranks import shard
    costs = [w.cell_modes() for w in I.batched_scan()]
    parts = shard(costs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) / (sum(costs) / world) < 1.02


def test_single_rank_is_a_no_op(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2609_03550_b300.ranks import Ranks, job_throughput
    r = Ranks(backend="gloo")
    r.barrier()
    assert r.world == 1 and r.max(3.5) == 3.5
    assert job_throughput(10.0, 2.0) == 5.0
