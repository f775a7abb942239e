"""Multi-process host logic of the replica runs, on CPU with gloo (world 2):
the job time is the slowest rank's and the work is the sum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2111_08666_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert replicas.rank_info() == (rank, world, rank)
    replicas.barrier()
    units, sec = replicas.aggregate(1000.0 * (rank + 1), 0.5 + rank)
    out[rank] = (units, sec)
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            assert out[r] == (3000.0, 1.5)


def test_aggregate_single_process_is_identity():
    assert replicas.aggregate(12.0, 3.0) == (12.0, 3.0)
