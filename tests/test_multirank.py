"""The multi-rank path of bench.py on CPU (gloo, world size 2): process-group
set-up from the launcher's environment, the barrier around the timed
region, and the maximum of the per-rank step times that the whole-job value
divides by.  A single transform does not shard (replicas only), so there is
no data-path collective to test; ranks that fail to join are covered by the
process group's own timeout."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist

    import bench
    r, local, w = bench._dist_init()
    assert (r, local, w) == (rank, rank, world)
    bench._barrier(w)
    # rank r "took" 1 + r seconds: every rank must see the slowest
    out[rank] = bench._max_over_ranks(1.0 + rank, w)
    bench._barrier(w)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_share_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world,
                           start_method="spawn", join=True)
        assert dict(out) == {0: 2.0, 1: 2.0}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench._max_over_ranks(3.5, 1) == 3.5
    bench._barrier(1)
