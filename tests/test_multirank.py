"""Multi-GPU path of bench.py on the host: under torchrun every rank advances its own ensemble
(stream_id = rank; the ensembles of different cases need no exchange) and the timing is the
maximum over ranks.  Checked with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from paper_2404_19602_gb300 import workloads as W

    t = bench.max_over_ranks(10.0 + rank, "cpu")
    p = bench.rank_workload(W.GAP_UQ_1E6, rank)
    o = O.Oracle(W.scaled(p, N=50))
    out[rank] = (t, p["stream_id"], float(o.state()[0, 0, 0]),
                 bench.throughput(1000, world, 10, 5, t))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 11.0                  # max over ranks
    assert (r0[1], r1[1]) == (0, 1)                 # one Philox stream per rank
    assert r0[2] != r1[2]                           # independent ensembles
    assert r0[3] == pytest.approx(1000 * 2 * 10 * 5 / 11e-3)  # whole-job particle-steps/s
