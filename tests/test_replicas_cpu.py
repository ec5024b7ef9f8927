"""Multi-GPU path on CPU: bench.py runs independent replicas (one suspension per
rank, no collective on the data path) and reports the steps of all ranks over
the slowest rank's time; checked here with two gloo ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip('torch')
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    elapsed = bench.max_over_ranks(1.0 + rank, dist, 'cpu')     # rank r took 1 + r seconds
    out[rank] = bench.replica_rate(world, 10, elapsed)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context('spawn')
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks agree: 2 ranks x 10 steps / max(1 s, 2 s)
    assert out[0] == out[1] == pytest.approx(10.0)
