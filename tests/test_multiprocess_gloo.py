"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1) run the replica
helpers of bench.py — barrier, max of the per-rank timings over ranks, and
the whole-job value summing all ranks' cells.  The RSST path itself is not
sharded (replicas only), so no collective touches the data."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), RSST_DIST_BACKEND="gloo")
    import bench
    w, r, _ = bench._dist()
    assert (w, r) == (world, rank)
    bench._barrier(w)
    t = 1.0 + rank                     # per-rank "time"
    tmax = bench._max_over_ranks(t, w)
    cells, steps = 1000, 5
    value = cells * 2 * steps * w / tmax
    out[rank] = (tmax, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1]
    tmax, value = out[0]
    assert tmax == 2.0
    assert value == pytest.approx(1000 * 2 * 5 * 2 / 2.0)
