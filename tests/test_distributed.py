"""The multi-rank bench path on CPU (gloo, world size 2): every rank works on
its own batch (its own seeded draw; no data-path collective, the test gathers
the batches only to check they differ); the job time is the slowest rank's
and the rate counts every rank's bytes."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch

    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms = bench.reduce_max_over_ranks(local_ms)
        value = bench.whole_job_gbs(1e9, world, ms)
        # each rank's own batch (a small one here); gathered only to check it
        x = bench.rank_input(rank, 4096)
        own = bool(torch.equal(x, synth.uniform(1, 4096, seed=1 + rank).reshape(-1)))
        parts = [torch.empty_like(x) for _ in range(world)]
        dist.all_gather(parts, x)
        distinct = all(not torch.equal(parts[i], parts[j]) for i in range(world) for j in range(i + 1, world))
        q.put((rank, ms, value, bench.env_rank(), own, distinct))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    results = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms, value, env, own, distinct in results:
        assert ms == pytest.approx(15.0)               # the slowest rank's time
        assert value == pytest.approx(2 * 1e9 / 15e-3 / 1e9)  # both ranks' bytes
        assert env == (rank, world, rank)
        assert own and distinct                        # its own seeded batch, unlike the other's


def test_single_process_reduction_is_identity():
    assert bench.reduce_max_over_ranks(3.5) == 3.5
    assert bench.whole_job_gbs(4e9, 1, 1.0) == pytest.approx(4000.0)
