"""The multi-GPU path (independent replicas per rank) on CPU with the gloo
backend, world size 2: each rank solves its own replica with the oracle and the
timing aggregation gives the slowest rank's time and the sum of all ranks' work."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_1108_5815_gb300 import inputs, replicas
        r, w, l = replicas.rank_info()
        assert (r, w, l) == (rank, world, rank)
        # every rank solves the same workload on its own (a replica)
        x, q = inputs.uniform_cube(600, 1234)
        phi, _ = O.Fmm(x, q, 4, 0.5, 16).evaluate()
        local_ms = 10.0 * (rank + 1)        # rank 1 is the slower one
        max_ms, units, rate = replicas.aggregate(local_ms, len(q))
        out.put((rank, max_ms, units, rate, float(np.sum(phi))))
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, max_ms, units, rate, checksum in res:
        assert max_ms == 20.0 and units == 1200
        assert rate == pytest.approx(1200 / 0.020)
    # identical replicas: identical results on both ranks
    assert res[0][4] == res[1][4]


def test_single_process_aggregate_is_identity():
    from paper_1108_5815_gb300 import replicas
    assert replicas.aggregate(5.0, 100) == (5.0, 100, 100 / 0.005)
