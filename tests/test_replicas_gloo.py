"""Host logic of multi-GPU replica runs, on CPU ranks over gloo (world size 2):
distinct seeds per rank, max-over-ranks time, whole-job throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1303_0270_gb300 import replicas
    r, w, lr = replicas.world()
    seconds = 1.0 + rank  # rank 1 is the slow one
    units = 100.0 * (rank + 1)
    out = {
        "world": (r, w, lr),
        "seed": replicas.rank_seed(1303, r),
        "max": replicas.max_over_ranks(seconds),
        "sum": replicas.sum_over_ranks(units),
        "tput": replicas.job_throughput(units, seconds),
    }
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_replica_bookkeeping_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0]["world"] == (0, 2, 0) and res[1]["world"] == (1, 2, 1)
    assert res[0]["seed"] != res[1]["seed"]
    for r in (0, 1):
        assert res[r]["max"] == 2.0
        assert res[r]["sum"] == 300.0
        assert res[r]["tput"] == pytest.approx(150.0)


def test_single_process_is_identity():
    from paper_1303_0270_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10.0, 2.0) == 5.0
