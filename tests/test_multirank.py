"""Host logic of the N > 1 benchmark path, on CPU with the gloo backend.

The shifted-solve path shards by independent problems: under torchrun each
rank runs its own replica (weak scaling) and the only cross-rank traffic is
the barrier around the timed region and the max-reduction of the timings.
This test runs that logic with world_size 2 on CPU processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import sys
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    t = 1.0 + rank            # rank 1 is the slowest
    tmax = bench.max_over_ranks(w, t)
    q.put((rank, w, local, tmax))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_barrier_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[3] == 2.0 for o in out)     # max over ranks seen by every rank
