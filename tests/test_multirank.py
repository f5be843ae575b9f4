"""The benchmark's multi-rank logic on CPU (gloo, world size 2): every rank
solves its own stack, timing is the maximum over ranks, and the value counts
all ranks' voxels."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, l = bench.dist_env()
    assert (w, r, l) == (world, rank, rank)
    bench.barrier(world)
    local_ms = 10.0 * (rank + 1)
    m = bench.reduce_max(local_ms, world)
    q.put((rank, m))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 20.0, 1: 20.0}


def test_single_rank_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5


def _leaving_worker(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    import bench
    bench.barrier(world)  # both ranks are up
    if rank == 1:
        # this rank leaves between steps, with nothing in flight
        q.put((rank, "left"))
        q.close()
        q.join_thread()
        os._exit(0)
    try:
        bench.barrier(world)  # the next step's barrier cannot complete
        msg = "no error"
    except Exception as e:  # the short process-group timeout (or the closed peer) ends it
        msg = "error: " + type(e).__name__
    q.put((rank, msg))
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_rank_leaving_is_detected_by_the_others():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got[1] == "left"
    assert got[0].startswith("error"), got
