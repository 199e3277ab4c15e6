"""bench.py's multi-rank logic on CPU (gloo, world size 2): the envs partition
across ranks with no data exchange (each rank its own seed), the timed region
is the maximum over ranks, and the reference arm prints on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 * (rank + 1), world)
    bench.barrier(world)

    class A:
        steps, warmup = 2, 1
    buf = io.StringIO()
    with redirect_stdout(buf):
        if rank != 0:
            bench.run_reference(A, world, rank)
    q.put((rank, t, bench.rank_seed(rank), buf.getvalue()))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, o0), (r1, t1, s1, o1) = out
    assert t0 == t1 == 3.0          # max over ranks
    assert s0 != s1                 # disjoint env sets
    assert o1 == ""                 # only rank 0 reports
