"""Multi-rank logic of bench.py on CPU (gloo, world size 2).

Each rank computes its own independent product (rows of Z and separate
instances share nothing, Sec. 2.1), so the only cross-rank steps are the
barrier and the max over ranks of the timed region; the whole-job value is
every rank's units over the slowest rank's time.
"""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench.dist_info()
        bench.barrier(w)
        ms = 10.0 + 5.0 * r                  # rank 1 is slower
        mx = bench.max_over_ranks(w, ms)
        units = list(bench.shard(7, r, w))
        q.put((r, mx, units, bench.whole_job_value([1] * w, 2e12, mx)))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_timing_and_sharding():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]         # max over ranks
    assert out[0][2] + out[1][2] == list(range(7))      # disjoint, complete
    assert abs(len(out[0][2]) - len(out[1][2])) <= 1
    assert out[0][3] == pytest.approx(2 * 2e12 / 15e-3 / 1e12)


def test_shard_covers_every_unit_once():
    sys.path.insert(0, ROOT)
    import bench
    for count in (0, 1, 5, 512):
        for ws in (1, 2, 3, 8):
            got = [u for r in range(ws) for u in bench.shard(count, r, ws)]
            assert got == list(range(count))
