"""Multi-rank logic of bench.py on CPU (gloo, world size 2): ray sharding gives
each rank its own cameras, and the job time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, _ = bench._dist()
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    cams = bench.rank_cameras(rank)
    out[rank] = (ws, r, t, np.asarray(cams[0]["c2w"]).tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_distinct_cameras():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == 2 and out[1][0] == 2
    assert out[0][1] == 0 and out[1][1] == 1
    assert out[0][2] == 15.0 and out[1][2] == 15.0  # both ranks see the slowest rank's time
    assert not np.allclose(out[0][3], out[1][3])     # each rank renders its own cameras


def test_single_process_is_identity():
    import bench
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    assert bench.max_over_ranks(3.5) == 3.5
    assert len(bench.rank_cameras(0)) == 8
