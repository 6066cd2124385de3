"""The multi-rank path of bench.py (torchrun, one independent replica per rank): the
barrier and the max-over-ranks timing reduction, run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
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
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dev = torch.device("cpu")
    bench.barrier(tdist, dev)
    t = bench.max_over_ranks(1.5 + rank, tdist, dev)
    # each rank solves its own seeded replica: the workload seeds differ by rank
    wl = bench.workload("small", 3 + rank)
    out[rank] = (t, float(wl.centres[0, 0]))
    bench.barrier(tdist, dev)
    tdist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_to_the_maximum():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 1.5 + world - 1
    assert res[0][1] != res[1][1]


def test_single_rank_needs_no_process_group():
    import bench
    rank, world, local, td = bench.dist_init(1)
    assert (rank, world, local, td) == (0, 1, 0, None)
    assert bench.max_over_ranks(3.0, None, None) == 3.0
