"""The replica (N > 1) logic of bench.py on two CPU ranks over gloo: each
rank decodes its own data, the job time is the slowest rank's, launches add
up, and throughput counts every rank's bits."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 * (rank + 1)          # rank 1 is slower
    launches = 100 + rank
    ms_max, n = bench.reduce_over_ranks(dist, ms, launches, torch.device("cpu"))
    dist.barrier()
    q.put((rank, bench.rank_data_seed(rank), ms_max, n,
           bench.job_throughput(world, 64, 1_000_000, 5, ms_max)))
    dist.destroy_process_group()


def test_two_replicas_reduce_time_and_launches():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = {o[1] for o in out}
    assert len(seeds) == world                      # different data per replica
    for _, _, ms_max, n, thr in out:
        assert ms_max == 20.0                       # slowest rank
        assert n == 201                             # launches summed
        assert thr == pytest.approx(2 * 64 * 1_000_000 * 5 / 0.020 / 1e6)
