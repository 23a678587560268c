"""Host logic of the N > 1 bench path on CPU (gloo, world size 2).

The solve does not shard (replicas only): each rank solves its own system and the job's
time is the slowest rank's.  Checks the max-over-ranks reduction and that the reference
arm runs on rank 0 only, in two spawned processes rendezvousing on 127.0.0.1.
"""
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


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.0 + rank, 10.0 - rank]
        got = bench.max_over_ranks(local, dist, "cpu")
        dist.barrier()
        # reference arm: ranks other than 0 return without work
        class A:
            pass
        ref_rc = bench.run_reference(A(), rank, world) if rank != 0 else None
        q.put((rank, got, ref_rc))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, got, rc = q.get(timeout=120)
        out[rank] = (got, rc)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == [2.0, 10.0] and out[1][0] == [2.0, 10.0]
    assert out[1][1] == 0


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks([3.5], None, "cpu") == [3.5]
