"""Host logic of the multi-GPU path, on CPU: instance sharding and the job-wide timing
reduction, the latter with two gloo ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2404_10270_gb300 import workloads as W
from paper_2404_10270_gb300.sharding import combine_timing, shard_instances


def test_shards_cover_every_instance_once_and_balance():
    counts = [p.n_particles() for p in W.ensemble(n_instances=512)]
    for world in (1, 2, 3, 8):
        shards = shard_instances(counts, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(512))
        loads = [sum(counts[i] for i in s) for s in shards]
        # greedy largest-first: the spread is at most the largest instance
        assert max(loads) - min(loads) <= max(counts)
    assert shard_instances([5, 5, 5], 5)[3:] == [[], []]
    with pytest.raises(ValueError):
        shard_instances([1], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counts = [p.n_particles() for p in W.ensemble(n_instances=64)]
    mine = shard_instances(counts, world)[rank]
    ms = 10.0 + 5.0 * rank
    ps = float(sum(counts[i] for i in mine))
    q.put((rank, mine, combine_timing(ms, ps)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    counts = [p.n_particles() for p in W.ensemble(n_instances=64)]
    assert sorted(out[0][1] + out[1][1]) == list(range(64))
    for _, _, (ms, ps) in out:
        assert ms == 15.0
        assert ps == float(sum(counts))
