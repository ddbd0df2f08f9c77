"""The multi-rank host path on CPU: two gloo ranks take disjoint shot ranges
that together cover every (rank, step) block, and the step time is the
maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2311_03906_gb300.dist import max_over_ranks, shard_range  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        steps, per = 5, 1000
        mine = [shard_range(rank, world, per, k, steps) for k in range(steps)]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = max_over_ranks(1.0 + rank * 0.5)
        q.put((rank, gathered, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_overlap():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t in results:
        assert t == 1.5
        ranges = sorted(r for per_rank in gathered for r in per_rank)
        assert ranges[0][0] == 0
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0, "ranges must tile the shot axis"
        assert ranges[-1][1] == world * 5 * 1000


def test_shard_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard_range(2, 2, 10, 0, 1)
    assert max_over_ranks(3.0) == 3.0


def _sample_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from workloads import surface_code
        ref = oracle.Program(surface_code(3, 3, 0.01))
        steps, per = 3, 500
        mine = []
        for k in range(steps):
            a, b = shard_range(rank, world, per, k, steps)
            mine.append((a, ref.sample(5, a, b - a)))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        if rank == 0:
            q.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_ranks_records_concatenate_to_one_rank_run():
    """Each gloo rank samples its own shot ranges (the oracle stands in for
    a GPU); ordered by shot index, the ranks' records are exactly those of
    one rank sampling every shot: the sharded path needs no exchange."""
    import numpy as np
    import oracle
    from workloads import surface_code
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_sample_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pieces = sorted((a, recs) for per_rank in gathered for a, recs in per_rank)
    total = pieces[-1][0] + len(pieces[-1][1][0])
    whole = oracle.Program(surface_code(3, 3, 0.01)).sample(5, 0, total)
    for k in range(3):
        np.testing.assert_array_equal(np.concatenate([recs[k] for _, recs in pieces]), whole[k])
