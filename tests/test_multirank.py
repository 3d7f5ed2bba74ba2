"""The multi-rank bench path on CPU: two gloo ranks, each with its own seeded batch (no
collective on the data path), the slowest rank's time and the whole-job rate."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(world, backend="gloo")
    batch = bench.make_batch(r, n_signals=40)
    t = 1.0 + r                                   # rank 1 is the slow one
    tmax = bench.max_over_ranks(t, w)
    bench.barrier(w)
    rate = bench.whole_job_rate(batch["n_out"], w, 10, tmax)
    out.put((r, w, tmax, rate, int(batch["n_out"]), float(batch["flat"][:8].sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, rate0, n0, s0), (r1, w1, t1, rate1, n1, s1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert t0 == t1 == 2.0                        # both ranks see the slowest time
    assert s0 != s1                               # each rank draws its own signals
    assert rate0 == pytest.approx(n0 * 2 * 10 / 2.0)
