"""Multi-GPU use is replicas only (each rank solves its own instances, no collective on the data
path); the host side of that — rank environment, distinct inputs per rank, the maximum of the
timings over the ranks — runs here on CPU ranks with the gloo backend."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from synth import workload
    r, w, lr = bench.dist_env()
    ph = workload(2, instance=r)["phase"]
    vals = bench.max_over_ranks([1.0 + r, 10.0 - r, float(ph.sum())], "cpu")
    out.put((r, w, lr, vals, int(ph.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_cpu_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, v0, s0), (r1, w1, l1, v1, s1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert s0 != s1                      # each rank solves its own instance
    assert v0 == v1 == [2.0, 10.0, float(max(s0, s1))]
