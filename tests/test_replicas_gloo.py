"""Multi-process host logic of the replicas path (world_size 2, gloo on CPU).

The imaging path does not shard: N GPUs run N independent replicas, the timed
region is bracketed by barriers and the job's throughput is N x steps over the
slowest rank's time.  These tests drive that aggregation and the reference
arm's rank handling with real gloo process groups on 127.0.0.1.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
        dist.barrier()
        ms, value = bench.replica_aggregate(ms_local, 20, dist, ws, "cpu")
        dist.barrier()
        q.put((rank, ms, value, bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_replica_aggregate_takes_slowest_rank():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(ws, port, q), nprocs=ws, join=True, start_method="spawn")
    res = sorted(q.get() for _ in range(ws))
    for rank, ms, value, env in res:
        assert ms == pytest.approx(150.0)                 # MAX over ranks
        assert value == pytest.approx(ws * 20 / 0.150)    # whole-job iterations per second
        assert env == (ws, rank, rank)


def test_single_process_aggregate_is_local():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replica_aggregate(80.0, 8, None, 1)
    assert ms == 80.0 and value == pytest.approx(100.0)


def _ref_worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))

    class A:
        workload, steps, warmup = "C0", 1, 0
    if rank != 0:
        q.put((rank, bench.run_reference(A())))   # ranks other than 0 exit without work
    else:
        q.put((rank, 0))


def test_reference_arm_other_ranks_exit_without_work():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_ref_worker, args=(ws, port, q), nprocs=ws, join=True, start_method="spawn")
    assert sorted(q.get() for _ in range(ws)) == [(0, 0), (1, 0)]
