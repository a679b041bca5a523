"""The multi-GPU path is replicas only: every rank solves its own instance and
the job time is the maximum over ranks.  This checks that aggregation with
two gloo ranks on CPU (each rank runs the CPU oracle on its own seed)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import workloads as W
    from oracle.newton import newton
    p = W.make_problem(16, seed=rank)
    r = newton(p, tol=1e-8)
    local = 1.0 + rank          # a per-rank "elapsed time"
    tmax = bench.max_over_ranks(local, world)
    line = bench.aggregate(tmax, steps=2, world=world)
    q.put((rank, r.newton_iters, tmax, line))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[2] == 2.0 for r in res)                     # max over ranks
    assert all(r[3]["value"] == pytest.approx(2.0 / (2 * 2)) for r in res)
    assert all(r[1] > 0 for r in res)
