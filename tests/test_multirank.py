"""The N > 1 host logic of the benchmark on CPU: two gloo ranks (127.0.0.1) interleave over
the pose path without overlap, the job time is the maximum over ranks, and the reference arm
runs on rank 0 only (the other ranks exit 0 without work)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    pose = bench.pose_of(rank, ws, 120)
    poses = [pose(i) for i in range(90)]
    times = bench.max_over_ranks([1.0 + rank, 5.0 - rank], ws, "cpu")
    # the reference arm: rank 0 alone runs it; here rank 1 must return 0 without work
    ref_rc = None
    if rank == 1:
        import argparse
        ref_rc = bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, poses, times, ref_rc))


def test_two_ranks_interleave_and_take_the_max():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, poses, times, ref_rc = q.get(timeout=120)
        out[rank] = (poses, times, ref_rc)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    p0, p1 = out[0][0], out[1][0]
    assert set(p0).isdisjoint(p1)                       # no frame rendered twice
    assert sorted(set(p0) | set(p1)) == list(range(120))
    assert out[0][1] == out[1][1] == [2.0, 5.0]          # max over ranks, same on both
    assert out[1][2] == 0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    pose = bench.pose_of(0, 1, 7)
    assert [pose(i) for i in range(9)] == [0, 1, 2, 3, 4, 5, 6, 0, 1]
