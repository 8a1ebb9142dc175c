"""The multi-GPU bench path is replicas only (no exchange step): each rank decimates its
own cloud and the job reports all ranks' points over the slowest rank's time.  The rank
reductions are checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(1.5 + rank, "cpu")      # rank 1 is slower
    total = bench.sum_over_ranks(1000 * (rank + 1), "cpu")  # uneven clouds
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, slowest, total))


def test_replica_reductions_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, total in res:
        assert slowest == pytest.approx(2.5) and total == pytest.approx(3000)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.0, "cpu") == 3.0
    assert bench.sum_over_ranks(7, "cpu") == 7.0
