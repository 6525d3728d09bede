"""afmm_mul_rows: one product in row blocks (Sec. 2.1: row I of Z needs
row I of X and all of Y), the unit each GPU computes when a product is
split over GPUs.  On one GPU: the blocks, each computed from its rows of X
only, must equal the whole-product call bit for bit, and match the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

import afmm_inputs as W
from _helpers import desc_for, gpu_operands, oracle_rows, rel_fro, sample_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOAD = {"A": "caseA_n8192_e4m3", "B": "caseB_n4096_f32"}


@pytest.mark.parametrize("variant", [1, 7])
@pytest.mark.parametrize("n,blocks", [(1000, 2), (2304, 3)])
@pytest.mark.parametrize("case", ["A", "B"])
def test_row_blocks_equal_the_whole_product(case, n, blocks, variant):
    import bench
    from paper_1308_2400_gb300 import Plan
    from paper_1308_2400_gb300.afmm import afmm_mul_rows
    inst = W.make(WORKLOAD[case], n=n, seed=n + variant)
    X, Y = gpu_operands(inst)
    Zw = torch.empty((n, n), dtype=torch.float32, device="cuda")
    p = Plan(desc_for(inst, variant=variant))
    p(X, Y, Zw)
    p.sync()
    Zb = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
    for r0, r1 in bench.row_blocks(n, blocks):
        Xr = X[r0:r1].clone()                   # only this block's rows exist
        Zr = torch.full((r1 - r0, n), float("nan"), dtype=torch.float32, device="cuda")
        afmm_mul_rows(p, r0, r1, Xr, Y, Zr)
        p.sync()
        Zb[r0:r1] = Zr
    p.close()
    assert torch.equal(Zb, Zw)
    rows = sample_rows(n, 12)
    assert rel_fro(Zb.cpu().numpy()[rows], oracle_rows(inst, rows)) <= 1e-6


def test_row_block_arguments_are_checked():
    from paper_1308_2400_gb300 import AfmmError, Plan
    from paper_1308_2400_gb300.afmm import (AFMM_ERR_INVALID_ARG, AFMM_ERR_UNSUPPORTED,
                                            afmm_mul_rows)
    inst = W.make("caseA_n8192_e4m3", n=600, seed=1)
    X, Y = gpu_operands(inst)
    Z = torch.empty((600, 600), dtype=torch.float32, device="cuda")
    p = Plan(desc_for(inst, variant=1))
    for r0, r1 in ((-1, 10), (10, 5), (0, 601)):
        with pytest.raises(AfmmError) as e:
            afmm_mul_rows(p, r0, r1, X, Y, Z)
        assert e.value.status == AFMM_ERR_INVALID_ARG
    with pytest.raises(AfmmError) as e:
        afmm_mul_rows(p, 0, 10, np.ascontiguousarray(inst.X), Y, Z)
    assert e.value.status == AFMM_ERR_INVALID_ARG
    afmm_mul_rows(p, 5, 5, X, Y, Z)              # empty block: nothing to do
    p.close()
    q = Plan(desc_for(inst, variant=0))          # CUDA-core form: whole products only
    with pytest.raises(AfmmError) as e:
        afmm_mul_rows(q, 0, 10, X, Y, Z)
    assert e.value.status == AFMM_ERR_UNSUPPORTED
    q.close()
