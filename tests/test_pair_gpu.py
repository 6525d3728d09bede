"""The two-SM split kernel (tcgen05 cta_group::2, 256 x 256 tiles per CTA
pair) and the exact form at sizes with several K chunks, against the
oracle (Sec. 2 loops, FP64 / int64).

From n = 512 the split form runs on CTA pairs; these sizes put partial pair
tiles at the edges (n not a multiple of 256) and single-tile problems.  The
same inputs through the one-CTA kernel (AFMM_TC_PAIR=0 at plan creation)
must agree with it within the tensor-core element bound, and the
host-buffer pipeline, which multiplies row blocks, must too.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import afmm_inputs as W
from _helpers import FP32_REL_FRO, rel_fro, run_gpu, sample_rows
from test_parity_gpu import check_fp32, tc_elem_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOAD = {"A": "caseA_n8192_e4m3", "B": "caseB_n4096_f32"}


@pytest.mark.parametrize("n", [512, 515, 777, 1000, 2049])
@pytest.mark.parametrize("case", ["A", "B"])
def test_pair_kernel_matches_the_oracle(case, n):
    inst = W.make(WORKLOAD[case], n=n, seed=n)
    Z, info = run_gpu(inst, variant=1)
    assert info["variant"] == 1
    check_fp32(inst, Z, sample_rows(n, 24), bound_fn=tc_elem_bound)


@pytest.mark.parametrize("case", ["A", "B"])
def test_pair_and_one_cta_kernels_agree(case, monkeypatch):
    n = 1283
    inst = W.make(WORKLOAD[case], n=n, seed=3)
    Zp, _ = run_gpu(inst, variant=1)
    monkeypatch.setenv("AFMM_TC_PAIR", "0")
    Z1, _ = run_gpu(inst, variant=1)
    rows = sample_rows(n, 32)
    bound = tc_elem_bound(inst, rows)
    assert np.all(np.abs(Zp[rows].astype(np.float64) - Z1[rows]) <= 2 * bound)
    check_fp32(inst, Zp, rows, bound_fn=tc_elem_bound)


@pytest.mark.parametrize("case", ["A", "B"])
def test_pair_kernel_host_buffers_pipelined(case):
    """Host X, Y, Z: the call pipelines copies with row blocks of the
    product, each block a pair-kernel launch over a range of rows."""
    from _helpers import desc_for
    from paper_1308_2400_gb300 import Plan
    n = 2304
    inst = W.make(WORKLOAD[case], n=n, seed=8)
    Xh = np.ascontiguousarray(inst.x_store if inst.x_store is not None else inst.X)
    Yh = np.ascontiguousarray(inst.y_store if inst.y_store is not None else inst.Y)
    Zh = np.full((n, n), np.nan, dtype=np.float32)
    p = Plan(desc_for(inst, variant=1))
    p(Xh, Yh, Zh)
    p.sync()
    p.close()
    check_fp32(inst, Zh, sample_rows(n, 24), bound_fn=tc_elem_bound)


@pytest.mark.parametrize("n", [512, 777, 1283])
@pytest.mark.parametrize("case", ["A", "B"])
def test_exact_form_many_chunks_is_bit_exact(case, n):
    """The exact form with int8 Base values at the extremes and u8
    Rep-factors up to 255: K chunks of 16 k-blocks, so every tile adds
    several chunks into Z in int32; the result must equal the oracle's
    integers."""
    from _helpers import oracle_rows
    rng = np.random.default_rng(n)
    base = rng.choice(np.array([-127, -126, 0, 1, 126, 127], dtype=np.int8), size=(n, n))
    rep = rng.integers(0, 256, size=(n, n)).astype(np.uint8)
    rep[rng.random((n, n)) < 0.3] = 0
    X, Y = (base, rep) if case == "A" else (rep, base)
    inst = W.Instance(case, X, Y, x_dtype="i8" if case == "A" else "u8",
                      y_dtype="u8" if case == "A" else "i8", z_dtype="i32", target="exact")
    from _helpers import torch_of
    from paper_1308_2400_gb300 import Plan, make_desc
    Z = torch.full((n, n), -7, dtype=torch.int32, device="cuda")
    p = Plan(make_desc(n, case, inst.x_dtype, inst.y_dtype, "i32", "exact", variant=5,
                       rep_max=255.0, base_max=127.0))
    assert p.info["k_split"] > 1 or n <= 512
    p(torch_of(X), torch_of(Y), Z)
    p.sync()
    p.close()
    rows = sample_rows(n, 40)
    R = oracle_rows(inst, rows)
    assert np.array_equal(Z.cpu().numpy()[rows].astype(np.int64), R)


@pytest.mark.parametrize("variant", [1, 7])
@pytest.mark.parametrize("case", ["A", "B"])
def test_pinned_host_buffers_pipelined(case, variant):
    """Pinned (page-locked) host X, Y, Z through the copy pipeline (row
    blocks of X in, products, row blocks of Z out, on three streams), two
    calls on one plan; the result must match the oracle as on device
    buffers."""
    from _helpers import desc_for
    from paper_1308_2400_gb300 import Plan
    n = 2304
    inst = W.make(WORKLOAD[case], n=n, seed=21 + variant)
    Xs = inst.x_store if inst.x_store is not None else inst.X
    Ys = inst.y_store if inst.y_store is not None else inst.Y
    Xh = torch.from_numpy(np.ascontiguousarray(Xs)).pin_memory()
    Yh = torch.from_numpy(np.ascontiguousarray(Ys)).pin_memory()
    Zh = torch.full((n, n), float("nan"), dtype=torch.float32).pin_memory()
    p = Plan(desc_for(inst, variant=variant))
    for _ in range(2):                       # the second call reuses the plan's buffers
        Zh.fill_(float("nan"))
        p(Xh, Yh, Zh)
        p.sync()
    p.close()
    Z = Zh.numpy()
    from test_fp8_gpu import fp8_elem_bound
    check_fp32(inst, Z, sample_rows(n, 24),
               bound_fn=tc_elem_bound if variant == 1 else fp8_elem_bound)
