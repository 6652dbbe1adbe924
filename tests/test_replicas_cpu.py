"""Multi-rank host logic on CPU: two gloo ranks shard frames with no
data-path collective and agree on the max of their step times."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2504_05148_gb300 import replicas


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_2504_05148_gb300 import scenes
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = replicas.rank_env()
        seeds = replicas.frame_seeds(r, 2, base=1000)
        outs = [oracle.compute(scenes.tiny(sd).left, scenes.tiny(sd).right, scenes.tiny(sd).lidar, 64,
                               dumps=False).out for sd in seeds]
        replicas.barrier()
        mx = replicas.max_over_ranks(1.5 + r)          # each rank reports its own "time"
        q.put((r, w, seeds, [int(o.sum()) for o in outs], mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_reduce_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, w0, s0, c0, m0), (r1, w1, s1, c1, m1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert not set(s0) & set(s1)                  # disjoint frames
    assert m0 == m1 == 2.5                        # max over ranks
    assert c0 != c1                               # different frames, different results


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.25) == 3.25
    assert replicas.frame_seeds(0, 3) == [2000, 2001, 2002]
    with pytest.raises(ValueError):
        replicas.frame_seeds(0, 5000)
