"""The multi-GPU path of bench.py is replicas only: every rank matches its own
pairs and the only collective is a max over ranks of the timed region.  Its
rank logic is checked here with world_size-2 gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 * (rank + 1), world)
    seeds = bench.rank_seeds(rank, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out.put((rank, t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_disjoint_pairs():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, gathered in res:
        assert t == 20.0                                  # the max over ranks, on every rank
        assert not set(gathered[0]) & set(gathered[1])    # each rank has its own pairs


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    a = type("A", (), dict(gpus=2, steps=1, warmup=0, cpu_pairs=1))()
    assert bench.run_reference(a) == 0
    assert capsys.readouterr().out == ""
