"""The benchmark's multi-rank bookkeeping (one replica per rank, no data
exchange; the job's time is the slowest rank's) on world size 2 with the
gloo backend on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init("gloo")
    t = 1.0 + 0.5 * r                       # rank 1 is the slow one
    bench.barrier(w)
    t_max = bench.max_over_ranks(t, w, device="cpu")
    out[r] = (w, local, t_max, bench.job_value(w, 20, t_max))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        w, local, t_max, value = out[r]
        assert w == 2 and local == r
        assert t_max == pytest.approx(1.5)
        assert value == pytest.approx(2 * 20 / 1.5)


def test_reference_arm_other_ranks_exit_without_work():
    """Under a multi-rank launch the oracle arm runs on rank 0 only: another
    rank exits 0 at once and prints nothing."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
