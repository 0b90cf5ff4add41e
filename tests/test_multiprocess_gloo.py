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


def test_two_rank_launch_prints_one_line_from_rank_zero():
    """bench.py launched the way multi-GPU runs are launched (torch.distributed.run,
    two ranks, 127.0.0.1), here on gloo with the CPU oracle arm: rank 0 alone
    prints the one JSON line and every rank exits 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RSST_DIST_BACKEND="gloo", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
