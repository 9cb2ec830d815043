"""Multi-rank (replica) logic of bench.py on CPU: two gloo ranks.  The job's
time is the slowest rank's, the whole-job rate counts every replica's cells,
and only rank 0 prints the reference arm's line."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    import bench
    elapsed = 1.0 + rank                       # rank 1 is the slower replica
    m = bench.max_over_ranks(elapsed, world)
    rate = bench.whole_job_rate(4096 * 5, world, m)

    class A:                                   # the reference arm's arguments
        gpus, steps, warmup = world, 1, 0

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A, rank) if rank != 0 else None
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as fh:
        json.dump({"max": m, "rate": rate, "printed": buf.getvalue()}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["max"] == 2.0                 # both ranks see the slowest time
        assert r["rate"] == 4096 * 5 * 2 / 2.0
    assert res[1]["printed"] == ""             # a non-zero rank of the reference arm does no work


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(100, 1, 2.0) == 50.0
