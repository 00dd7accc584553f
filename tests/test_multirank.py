"""N > 1 host logic on the CPU: two gloo ranks shard streams and reduce the timing.

Each rank takes its stream range from ``sharding.rank_seeds``, generates it with
the oracle (the GPU path is the same call per rank), and the ranks check that
(a) their ranges are disjoint and together cover the streams a single process
would generate, (b) concatenating their outputs equals one process generating
all streams, and (c) the timing reduction returns the max over ranks.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle as O
    from paper_2405_19493_gb300 import sharding

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 8
        seeds = sharding.rank_seeds(rank, world, n)
        out, _, _ = O.generate("splitmix64", "zig128", seeds, uniform_len=64)
        t = torch.from_numpy(out)
        gathered = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(gathered, t)
        sd = torch.from_numpy(seeds.view(np.int64))
        gs = [torch.empty_like(sd) for _ in range(world)]
        dist.all_gather(gs, sd)
        mx = sharding.max_over_ranks(10.0 + rank, dist)
        if rank == 0:
            q.put((torch.cat(gathered).numpy(), torch.cat(gs).numpy().view(np.uint64), mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_matches_single_process():
    import torch.multiprocessing as mp

    from paper_2405_19493_gb300 import sharding, workloads
    import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out, seeds, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.array_equal(seeds, workloads.seeds(16))
    single, _, _ = O.generate("splitmix64", "zig128", workloads.seeds(16), uniform_len=64)
    assert np.array_equal(out, single)
    assert mx == 11.0
    assert sharding.rank_streams(1, 2, 8) == (8, 16)
    with pytest.raises(ValueError):
        sharding.rank_streams(2, 2, 8)
