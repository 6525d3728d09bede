"""One product split by row blocks over ranks, on CPU (gloo, world size 2).

Row I of Z is final after the K loop of row I and needs only row I of X
and all of Y (Sec. 2.1), so a product splits into row blocks of X and Z
with Y copied to every rank.  Each rank computes its block with the oracle
(the Sec. 2 loops); rank 0 gathers the blocks, and their concatenation must
equal the oracle's whole product bit for bit.  The block boundaries come
from bench.row_blocks, the partition the --shard rows mode uses.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, n, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import afmm_inputs as W
    import bench
    from oracle import afmm_case_a
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        inst = W.make("caseA_n8192_e4m3", n=n, seed=4)
        # Y from rank 0 to every rank: the exchange of the row split.
        Y = torch.from_numpy(inst.Y.astype(np.int64)) if rank == 0 else \
            torch.empty((n, n), dtype=torch.int64)
        dist.broadcast(Y, src=0)
        r0, r1 = bench.row_blocks(n, ws)[rank]
        Xb = np.zeros((n, n), dtype=inst.X.dtype)
        Xb[r0:r1] = inst.X[r0:r1]                      # this rank holds its rows only
        Zr, _ = afmm_case_a(Xb, Y.numpy(), (r0, r1))
        rows = torch.zeros((max(b - a for a, b in bench.row_blocks(n, ws)), n),
                           dtype=torch.float64)
        rows[: r1 - r0] = torch.from_numpy(Zr)
        got = [torch.zeros_like(rows) for _ in range(ws)] if rank == 0 else None
        dist.gather(rows, got, dst=0)
        if rank == 0:
            parts = [g[: b - a].numpy() for g, (a, b) in zip(got, bench.row_blocks(n, ws))]
            Z = np.concatenate(parts, axis=0)
            full, _ = afmm_case_a(inst.X, inst.Y)
            q.put(("ok", bool(np.array_equal(Z, full)), Z.shape))
        else:
            q.put(("rank1", True, None))
    finally:
        dist.destroy_process_group()


def test_row_blocks_concatenate_to_the_oracle_product():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + (os.getpid() % 1000)
    n = 300
    ps = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=180) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = [o for o in out if o[0] == "ok"][0]
    assert res[1] is True and res[2] == (n, n)


def test_row_blocks_partition():
    sys.path.insert(0, ROOT)
    import bench
    for n in (0, 1, 255, 256, 300, 8192, 8193):
        for ws in (1, 2, 3, 8):
            b = bench.row_blocks(n, ws)
            assert len(b) == ws and b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(ws - 1))
            assert all(r0 % 256 == 0 for r0, _ in b if r0 < n)
            sizes = [r1 - r0 for r0, r1 in b]
            assert max(sizes) - min(sizes) <= 2 * 256 - 1     # one unit, plus the short tail
