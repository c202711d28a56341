"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.  One
OS-MPM instance does not shard (multiplicative Schwarz solves its two
subdomains one after the other), so N GPUs run N independent replicas; the
only cross-rank steps are the barrier, the max of the per-rank times and the
sum of the per-rank units.  No collective touches the data path."""
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


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, local, w = bench.dist_init(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    t_max = bench.max_over_ranks(1.0 + rank, w)        # rank 1 is the slow one
    units = bench.sum_over_ranks(100.0 * (rank + 1), w)
    out[rank] = (t_max, units)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_reduction_of_time_and_units():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == (2.0, 300.0) and out[1] == (2.0, 300.0)


def _ref_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, local, w = bench.dist_init(world)
    calls = []
    bench.oracle_sample = lambda n: (calls.append(n), (0.5, 10.0))[1]
    bench.oracle_instance_sample = lambda i, s: (calls.append((i, s)), (0.5, 10.0))[1]

    class A:
        steps, warmup = 2, 1
        workload = "default"
    res = bench.run_reference(A, r, w)
    out[rank] = (res is None, len(calls), None if res is None else res["value"])
    import torch.distributed as dist
    dist.destroy_process_group()


def test_reference_arm_runs_on_rank0_only():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_ref_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[1] == (True, 0, None)
    assert out[0][0] is False and out[0][1] == 3 and out[0][2] == pytest.approx(20.0)
