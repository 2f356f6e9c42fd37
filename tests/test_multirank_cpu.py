"""The N > 1 path of bench.py on CPU: two gloo ranks, launched the way the
benchmark's replicas are (RANK / WORLD_SIZE / MASTER_ADDR from the environment).
Each rank advances its own seeded level (weak scaling, no data-path
collective); the only collective is the max over ranks of the timed region."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w = bench.dist_init(backend="gloo")
    assert (r, w) == (rank, world)
    # the slowest replica's time is the job's time
    t = bench.max_over_ranks(10.0 + rank, w)
    bench.barrier(w)
    sizes, offsets, flat = bench.build_level(r, npatch=5)
    got = [None] * w
    dist.all_gather_object(got, (np.asarray(sizes).tolist(), float(sum(f.sum() for f in flat))))
    dist.destroy_process_group()
    out.put((rank, t, got))


def test_two_gloo_ranks_run_independent_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, got in res:
        assert t == 11.0                      # max over ranks of 10 + rank
        (sz0, sum0), (sz1, sum1) = got
        assert sz0 == sz1                     # same patch shapes on every rank
        assert sum0 != sum1                   # each rank its own seeded realisation
