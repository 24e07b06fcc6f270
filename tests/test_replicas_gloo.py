"""The multi-rank (replica) path on CPU: two gloo ranks, disjoint shards, max timing."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_08510_gb300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1904_08510_gb300.workload import make_batch
    ws, rk, _ = R.dist_info()
    ncol = 3
    b = make_batch("ragged", ncol, R.shard_seed(100, rk, ncol), n_range=(32, 96))
    r = O.solve(b, O.default_params(precond=2), threads=1)
    t = 1.0 + rk                       # a per-rank "time"
    tmax = R.max_over_ranks(t)
    dist.barrier()
    q.put((rk, ws, tmax, b.col_off.tolist(), r["ne"].tolist(), int((r["status"] == 0).sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_shards_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=120) for _ in range(2)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, off0, ne0, ok0), (r1, w1, t1, off1, ne1, ok1) = got
    assert (w0, w1) == (2, 2) and t0 == t1 == 2.0
    assert ok0 == ok1 == 3
    # the two shards are different columns, and each equals a single-process solve
    import oracle as O
    from paper_1904_08510_gb300.workload import make_batch
    b1 = make_batch("ragged", 3, R.shard_seed(100, 1, 3), n_range=(32, 96))
    r1 = O.solve(b1, O.default_params(precond=2), threads=1)
    assert np.array_equal(np.array(ne1), r1["ne"])
    assert off0 != off1 or ne0 != ne1
    assert R.job_throughput(3, 2, 5, 2.0) == pytest.approx(15.0)
