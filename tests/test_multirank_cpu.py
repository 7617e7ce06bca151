"""Host-side logic of the multi-GPU run, on CPU with two gloo ranks: each rank
times its own replica; the job's time is the maximum over ranks and its
throughput counts every rank's queries; ranks draw different queries."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1506_08620_gb300 import workloads as W
    t = bench.max_over_ranks(1.0 + 2.5 * rank, dist)
    dist.barrier()
    seed = bench.rank_seed(W, 2, rank)
    w = W.workload2(n_knots=1025, m=64, seed=seed)
    q.put((rank, t, seed, w["Z"][:4].tolist()))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_distinct_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == pytest.approx(3.5)
    assert res[0][2] is None and res[1][2] is not None
    assert res[0][3] != res[1][3]


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(4.25) == 4.25
