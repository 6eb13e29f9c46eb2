"""The benchmark's rank logic with two gloo ranks on the CPU: the barrier,
the max over ranks of the per-rank times and the whole-job throughput (weak
scaling, no data-path collective)."""
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
    from paper_2609_03550_b300.ranks import Ranks, job_throughput
    r = Ranks(backend="gloo")
    r.barrier()
    t = 1.0 + rank  # rank 1 is the slowest
    tmax = r.max(t)
    value = job_throughput(100.0, r.world, tmax)
    r.barrier()
    q.put((rank, r.world, tmax, value))
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
    for _, w, tmax, value in out:
        assert w == 2 and tmax == 2.0
        assert value == pytest.approx(2 * 100.0 / 2.0)


def test_single_rank_is_a_no_op(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2609_03550_b300.ranks import Ranks, job_throughput
    r = Ranks(backend="gloo")
    r.barrier()
    assert r.world == 1 and r.max(3.5) == 3.5
    assert job_throughput(10.0, 1, 2.0) == 5.0
