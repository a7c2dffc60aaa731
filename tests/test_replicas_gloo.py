"""Host logic of the multi-GPU bench path on CPU: two gloo ranks, as torchrun would start them.

The decoder does not shard one stream (blocks are independent but the one-pass and wavefront kernels
already spread one stream over the whole GPU), so N GPUs run N replicas, each decoding its own stream, and
the step time is the maximum over ranks.  These tests check that reduction and the per-rank workload
choice without a GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    try:
        w, r, local = bench.dist_setup()
        ms = 10.0 + 5.0 * r                       # rank 1 is the slower replica
        q.put((r, w, local, bench.max_over_ranks(ms, w, "cpu"), bench.stream_seed("text", r)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step_and_distinct_streams():
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
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == pytest.approx(15.0) for r in res)      # every rank sees the maximum
    assert res[0][4] != res[1][4]                               # each replica decodes its own stream


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    os.environ.pop("WORLD_SIZE", None)
    assert bench.dist_setup()[0] == 1
