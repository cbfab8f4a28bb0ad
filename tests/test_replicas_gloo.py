"""The multi-GPU form is replicas only (one independent snapshot per rank, no
exchange step in the method): what bench.py adds for N > 1 is bookkeeping --
the rendezvous, a barrier around the timed steps, the maximum of the ranks'
step times, and a distinct snapshot per rank.  This runs that bookkeeping as
two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    step_ms = 3.0 + rank  # rank 1 is the slower one
    out[rank] = (bench.max_over_ranks(w, step_ms), tuple(bench.rank_seeds(r)))
    bench.barrier(w)
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="the CPU (gloo) form of the multi-rank bookkeeping")
def test_two_gloo_ranks_agree_on_the_slowest_step():
    world = 2
    with mp.get_context("spawn").Manager() as m:  # no fork of a multi-threaded process
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    # both ranks report the slowest rank's time (the bench's whole-job clock)
    assert res[0][0] == res[1][0] == 4.0
    # independent replicas: each rank reduces its own snapshot
    assert res[0][1] != res[1][1]
    assert res[0][1] == (10, 11, 12, 13)
