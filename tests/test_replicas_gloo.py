"""Multi-rank replica logic on CPU with the gloo backend (world size 2).

Each rank solves its own seeded batch (no collective on the data path); only
the timing (max over ranks) and the solve counts (sum over ranks) cross
ranks.  Checked here without a GPU: the reductions, the whole-job value and
that the ranks' batches differ.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2604_22625_gb300 import replicas, synthetic  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = replicas.dist_env()
    assert (ws, r) == (world, rank)
    seconds = 1.0 + rank          # rank 1 is the slow one
    units = 10.0 * (rank + 1)
    value, t, u = replicas.job_throughput(dist, units, seconds)
    probs = synthetic.config_batch(seed=replicas.rank_seed(3, rank), n_single=2, n_multi=0)
    out[rank] = (value, t, u, float(probs[0].alpha[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    v0, t0, u0, a0 = out[0]
    v1, t1, u1, a1 = out[1]
    assert t0 == t1 == 2.0 and u0 == u1 == 30.0
    assert v0 == v1 == 15.0
    assert a0 != a1                         # each rank has its own batch


def test_single_process_is_identity():
    assert replicas.job_throughput(None, 12.0, 3.0) == (4.0, 3.0, 12.0)
    assert replicas.rank_seed(3, 0) == 3
