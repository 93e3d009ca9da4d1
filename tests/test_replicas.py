"""The multi-GPU replica bookkeeping on CPU with two gloo ranks: disjoint
frames per rank, the maximum of the ranks' times, the job's rate."""
import os
import socket

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


def _rank_main(rank, world, port, out):
    from paper_1310_1371_gb300 import replicas as R
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert R.env_rank() == (rank, rank, world)
    seeds = R.frame_seeds(rank, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    dist.barrier()
    t = R.max_over_ranks(1.5 + rank, dist)           # the slowest rank's time
    rate = R.job_rate(4, world, t)
    out[rank] = (gathered, t, rate)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a threaded process
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        gathered, t, rate = res[rank]
        flat = [tuple(s) for g in gathered for s in g]
        assert len(flat) == 8 and len(set(flat)) == 8          # no frame on two ranks
        assert t == 1.5 + (world - 1)                           # max over ranks
        assert rate == pytest.approx(4 * world / t)             # all ranks' frames / slowest time


def test_single_process_defaults():
    from paper_1310_1371_gb300 import replicas as R
    assert R.max_over_ranks(3.0) == 3.0
    assert R.job_rate(96, 1, 2.0) == 48.0
    assert R.frame_seeds(0, 2) == [[1002, 0], [1002, 1]]
