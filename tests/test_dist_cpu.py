"""The multi-rank path of bench.py on CPU: two gloo ranks, barrier and the
max-over-ranks timing reduction (replicas only: no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local, pg = bench.dist_setup()
    assert (r, w) == (rank, world) and pg is not None
    bench.barrier(pg)
    mx = bench.allreduce(pg, 10.0 + rank, "max")
    sm = bench.allreduce(pg, 1.0 + rank, "sum")
    out[rank] = (mx, sm)
    pg.destroy_process_group()


def test_two_gloo_ranks_time_as_the_slowest():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == (11.0, 3.0) and out[1] == (11.0, 3.0)


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
