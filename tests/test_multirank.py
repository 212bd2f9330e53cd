"""The benchmark's multi-rank path on CPU: two gloo ranks (one process per
GPU in production).  Instances shard with no data-path collective: every
rank draws its own seeded batch of the same shape, the job's time is the
slowest rank's (an all-reduce MAX, the only collective) and the job's rate
is the units of all ranks over that time."""
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


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, _ = bench.dist_env()
    prob, b = bench.workload(r)
    t_local = 1.0 + 0.5 * r                  # a slower second rank
    t_max = bench.max_over_ranks(t_local, w, "cpu")
    out[rank] = (w, r, b.x0.copy(), b.T.copy(), t_max, bench.job_throughput(b.x0.shape[0], t_max, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_collectives():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    (w0, r0, x0a, Ta, tm0, v0), (w1, r1, x0b, Tb, tm1, v1) = out[0], out[1]
    assert (w0, r0, w1, r1) == (2, 0, 2, 1)
    # weak scaling: same batch size, different seeded instances
    assert x0a.shape == x0b.shape and Ta.shape == Tb.shape
    assert not np.array_equal(x0a, x0b)
    # the slowest rank's time on every rank, and the job rate from it
    assert tm0 == tm1 == 1.5
    assert v0 == v1 == pytest.approx(2 * x0a.shape[0] / 1.5)
