"""Multi-GPU path of bench.py on CPU: level solves are independent, so N
GPUs are N replicas with different seeds (weak scaling) and the only
collective is the max over ranks of the timed region.  Checked here with two
gloo ranks on 127.0.0.1 (no GPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads as W

    seed = bench.replica_seed(rank)
    solves = W.ragged_batch(n_solves=3, seed=seed)
    m = bench.reduce_max(1.0 + rank, torch.device("cpu"))
    out[rank] = (seed, int(solves[0][0].n_oct), m)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_distinct_work_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    seeds = {out[r][0] for r in range(world)}
    assert len(seeds) == world                      # each rank has its own problems
    assert all(out[r][2] == float(world) for r in range(world))   # max over ranks seen by all


def test_reduce_max_without_process_group():
    import bench

    assert bench.reduce_max(3.5) == 3.5


def _failing_worker(rank, world, port, out):
    import datetime

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    import bench

    if rank == 1:
        out[rank] = "left"  # fails between steps: never joins the step's max-over-ranks
        os._exit(0)
    try:
        bench.reduce_max(1.0, torch.device("cpu"))
        out[rank] = "completed"
    except Exception as e:  # the collective ends with an error instead of waiting forever
        out[rank] = "error: " + type(e).__name__


@pytest.mark.timeout(120)
def test_a_rank_that_leaves_is_seen_by_the_others():
    """A replica that fails between steps: the remaining rank's timing
    collective (the only one of the replicas path) ends with an error after
    the process group's short timeout instead of hanging."""
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.start_processes(_failing_worker, args=(world, port, out), nprocs=world, join=False,
                             start_method="spawn")
    try:
        while not ctx.join(timeout=60):
            pass
    except Exception:
        pass  # a rank's exit is reported by join; the outcome is in `out`
    assert out.get(1) == "left"
    assert str(out.get(0, "")).startswith("error"), dict(out)
