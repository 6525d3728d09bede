"""Parity of the CUDA library with the CPU oracle (GPU tests).

Every product goes through the C ABI (the Python binding only marshals
arguments) and is compared element by element with the FP64 / int64 oracle
on the same seeded inputs:

* integer work is bit-exact;
* FP32-target variants meet the relative Frobenius bar 1e-6, and each
  element meets the rounding bound of the kernel's summation (derived in
  ``simt_f32_elem_bound``);
* FP64-target variants meet 1e-12 and an element bound of the slicing
  truncation plus recombination rounding.

Sizes span several tiles and ragged tails; at the workloads' full sizes the
oracle checks sampled rows.
"""
from __future__ import annotations

import numpy as np
import pytest

import afmm_inputs as W
from _helpers import (FP32_REL_FRO, FP64_REL_FRO, U32, U64, abs_product, desc_for,
                      gpu_operands, oracle_rows, rel_fro, run_gpu, sample_rows, torch_of)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIMT_BK = 32          # k block of the zero-skip CUDA-core kernel
DENSE_BK = 128        # k block of the dense CUDA-core kernel
RAGGED = [1, 2, 7, 33, 63, 65, 127, 129, 257, 300]


def simt_f32_elem_bound(inst, rows=None):
    """Worst-case rounding of the K-blocked FP32 sums, to first order.

    Each product is formed exactly by the FMA and rounded once when added;
    a k block sums at most b terms from zero (b = 32 in the zero-skip
    kernel, 128 in the dense one), then <= ceil(n/b) block sums are added
    to the running total: error <= (min(n, b) + ceil(n/b)) u32 sum|x y|
    for each element.  (min(n, 128) + ceil(n/32)) covers both kernels; the
    rounding of the real factor to FP32 (u32) when it arrives in FP64 and a
    unit of slack make the +2.
    """
    n = inst.n
    g = (min(n, DENSE_BK) + -(-n // SIMT_BK) + 2) * U32
    return g * abs_product(inst, rows) + 1e-30


def tc_elem_bound(inst, rows=None, slices=3):
    """Rounding of the tensor-core form, to first order.

    The slices of an FP32 value are exact (hi + mid + lo == x).  The hi
    products and the smaller slices' products go to two FP32 accumulators;
    each of the ceil(n/16) MMAs into either rounds at most once relative to
    that accumulator's sum|x y|, and the epilogue adds the two with one
    rounding.  The factor 2 allows a truncating accumulator.
    """
    g = 2 * (2 * -(-inst.n // 16) + 8) * U32
    return g * abs_product(inst, rows) + 1e-30


def check_fp32(inst, Z, rows=None, bound_fn=None):
    R = oracle_rows(inst, rows)
    Zs = Z if rows is None else Z[rows]
    assert np.all(np.isfinite(Zs))
    err = rel_fro(Zs, R)
    assert err <= FP32_REL_FRO, (inst.name, err)
    bound = (bound_fn or simt_f32_elem_bound)(inst, rows)
    bad = np.abs(Zs.astype(np.float64) - R) > bound
    assert not bad.any(), (inst.name, int(bad.sum()))
    return err


# ------------------------------------------------------------------ K1 FP32
@pytest.mark.parametrize("n", RAGGED)
@pytest.mark.parametrize("workload", ["caseB_n4096_f32", "caseA_n8192_e4m3"])
def test_simt_f32_ragged(workload, n):
    inst = W.make(workload, n=n, seed=n)
    Z, info = run_gpu(inst, variant=0)
    assert info["variant"] == 0
    check_fp32(inst, Z)


@pytest.mark.parametrize("n", [1, 65, 129, 300])
def test_simt_f32_skip_kernel_on_dense_data(n):
    """A low density hint picks the zero-skip kernel; on dense data it takes
    its all-k path and must give the same sums (hints never change Z)."""
    inst = W.make("caseA_n8192_e4m3", n=n, seed=n + 5)
    Z, _ = run_gpu(inst, variant=0, d1_hint=0.05)
    check_fp32(inst, Z)


@pytest.mark.parametrize("hints", [True, False])
def test_simt_f32_sparse_base_skips(hints):
    """Very sparse Base factor: whole 4-row groups are zero for most k.
    With its density hint (0.03) the zero-skip kernel runs; without hints
    the dense kernel does."""
    rng = np.random.default_rng(3)
    n = 515
    X = rng.uniform(-1, 1, size=(n, n)).astype(np.float32)
    X[rng.random((n, n)) > 0.03] = 0
    X[64:128] = 0                       # an all-zero 64-row tile
    Y = rng.integers(0, 10, size=(n, n)).astype(np.int32)
    inst = W.Instance("A", X, Y, name="sparse", x_dtype="f32", y_dtype="i32",
                      z_dtype="f32", target="fp32")
    Z, _ = run_gpu(inst, variant=0, hints=hints)
    check_fp32(inst, Z)
    assert np.all(Z[64:128] == 0)


def test_simt_f32_strided_operands():
    """Leading dimensions that are not multiples of 4 take the scalar loads
    and stores of both kernels."""
    from paper_1308_2400_gb300 import Plan, make_desc
    n, ld = 203, 207
    for d1 in (-1.0, 0.05):
        inst = W.make("caseA_n8192_e4m3", n=n, seed=11)
        X = torch.zeros((n, ld), dtype=torch.float32)
        X[:, :n] = torch.from_numpy(inst.X.astype(np.float32))
        Y = torch.zeros((n, ld), dtype=torch.uint8)
        Y[:, :n] = torch.from_numpy(inst.Y.astype(np.uint8))
        Z = torch.full((n, ld), float("nan"))
        X, Y, Z = X.cuda(), Y.cuda(), Z.cuda()
        plan = Plan(make_desc(n, "A", "f32", "u8", "f32", "fp32", variant=0,
                              d1=d1, ldx=ld, ldy=ld, ldz=ld))
        plan(X, Y, Z)
        plan.sync()
        plan.close()
        Zn = Z.cpu().numpy()
        check_fp32(inst, Zn[:, :n].copy())
        assert np.all(np.isnan(Zn[:, n:]))


def test_simt_f32_case_b_full_size_sampled():
    inst = W.make("caseB_n4096_f32")
    Z, _ = run_gpu(inst, variant=0)
    check_fp32(inst, Z, sample_rows(inst.n, 24))


def test_simt_f32_case_a_full_size_sampled():
    inst = W.make("caseA_n8192_e4m3")
    Z, _ = run_gpu(inst, variant=0)
    check_fp32(inst, Z, sample_rows(inst.n, 12))


# ------------------------------------------------------------------ tcgen05
TC_RAGGED = [1, 7, 33, 127, 128, 129, 255, 256, 257, 300, 513]


@pytest.mark.parametrize("n", TC_RAGGED)
@pytest.mark.parametrize("workload", ["caseA_n8192_e4m3", "caseB_n4096_f32"])
def test_tc_bf16x3_ragged(workload, n):
    inst = W.make(workload, n=n, seed=n + 1)
    Z, info = run_gpu(inst, variant=1)
    assert info["variant"] == 1 and info["slices"] == 3
    check_fp32(inst, Z, bound_fn=tc_elem_bound)


def _padded(arr, ld, dtype):
    """arr (n x n) in an n x ld buffer of torch dtype `dtype` (padding 0)."""
    n = arr.shape[0]
    buf = np.zeros((n, ld), dtype=np.float64)
    buf[:, :n] = arr
    if dtype == "e4m3":
        return torch.from_numpy(buf.astype(np.float32)).to(torch.float8_e4m3fn) \
            .view(torch.uint8).cuda()
    tdt = {"u8": torch.uint8, "i32": torch.int32, "f32": torch.float32,
           "bf16": torch.bfloat16}[dtype]
    return torch.from_numpy(buf.astype(np.float64)).to(tdt).cuda()


@pytest.mark.parametrize("n,yd,pad", [(512, "e4m3", 0), (520, "i32", 0), (600, "u8", 3),
                                      (777, "f32", 5), (1000, "bf16", 1), (1537, "e4m3", 16)])
@pytest.mark.parametrize("variant", [1, 10])
def test_tc_pair_case_a_storage_types_and_padding(variant, n, yd, pad):
    """Case A on the two-SM kernel (split BF16 and FP16 forms): ragged n,
    every Rep-factor storage type through the transposition, padded rows
    of X, Y (the per-element load paths) and Z (padding left alone)."""
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(n + pad)
    X = rng.uniform(-1, 1, size=(n, n))
    X[rng.random((n, n)) > 0.7] = 0
    X = X.astype(np.float32)
    Y = np.minimum(rng.poisson(3.0, size=(n, n)), 16).astype(np.int64)
    Y[:, -1] = 16                       # the last, partial tile column
    ld = n + pad
    Xt = _padded(X, ld, "f32")
    Yt = _padded(Y, ld, yd)
    Zb = torch.full((n, ld), 7.0, dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "A", "f32", yd, "f32", "fp32", variant=variant,
                       ldx=ld, ldy=ld, ldz=ld))
    p(Xt, Yt, Zb)
    p.sync()
    Z = Zb.cpu().numpy()
    inst = W.Instance("A", X, Y, name=f"mn_{yd}", x_dtype="f32", y_dtype=yd,
                      z_dtype="f32", target="fp32")
    check_fp32(inst, Z[:, :n], bound_fn=tc_elem_bound)
    assert np.all(Z[:, n:] == 7.0)


@pytest.mark.parametrize("n", [32, 200, 256, 1000])
def test_tc_fused_split_kernel(n):
    """Case A with the split done inside the product kernel
    (AFMM_FLAG_FUSED_SPLIT): same accuracy bar as the separate pass."""
    from paper_1308_2400_gb300.afmm import AFMM_FLAG_FUSED_SPLIT
    inst = W.make("caseA_n8192_e4m3", n=n, seed=n + 3)
    Z, info = run_gpu(inst, variant=1, flags=AFMM_FLAG_FUSED_SPLIT)
    check_fp32(inst, Z, bound_fn=tc_elem_bound)


def test_tc_bf16x3_case_a_full_size_sampled():
    inst = W.make("caseA_n8192_e4m3")
    Z, info = run_gpu(inst)                 # the planner's choice
    assert info["variant"] == 1
    check_fp32(inst, Z, sample_rows(inst.n, 12), bound_fn=tc_elem_bound)


def test_tc_bf16x3_case_b_full_size_sampled():
    inst = W.make("caseB_n4096_f32")
    Z, info = run_gpu(inst, variant=1)
    check_fp32(inst, Z, sample_rows(inst.n, 24), bound_fn=tc_elem_bound)


def test_tc_accumulation_is_exact_for_integers():
    """Integer operands whose partial sums stay below 2^24 must come out
    exact from the FP32 tensor-core accumulator (products are exact in
    FP32 and every partial sum is representable)."""
    rng = np.random.default_rng(21)
    n = 2048                            # |partial| <= 2048 * 255 * 16 < 2^24
    X = rng.integers(-255, 256, size=(n, n)).astype(np.float32)
    X[0, :] = 255.0
    Y = rng.integers(0, 17, size=(n, n)).astype(np.int32)
    Y[:, 0] = 16
    inst = W.Instance("A", X, Y, name="probe", x_dtype="f32", y_dtype="i32",
                      z_dtype="f32", target="fp32")
    Z, _ = run_gpu(inst, variant=1)
    R = X.astype(np.int64) @ Y.astype(np.int64)
    assert np.array_equal(Z.astype(np.int64), R)


def test_tc_two_slices_fall_short_of_fp32():
    """hi + lo BF16 keeps ~16 bits of each value: the error is well above
    the three-slice form and above the FP32 bar on this workload."""
    inst = W.make("caseA_n8192_e4m3", n=1024, seed=3)
    Z2, _ = run_gpu(inst, variant=2)
    Z3, _ = run_gpu(inst, variant=1)
    R = oracle_rows(inst)
    e2, e3 = rel_fro(Z2, R), rel_fro(Z3, R)
    assert 1e-6 < e2 < 1e-4 and e3 < 1e-6 and e2 > 4 * e3


def test_bounded_wait_times_out_and_context_survives():
    from paper_1308_2400_gb300.afmm import afmm_selftest_bounded_wait
    assert afmm_selftest_bounded_wait(50_000_000) == 7      # AFMM_ERR_TIMEOUT
    inst = W.make("caseA_n8192_e4m3", n=200, seed=4)
    Z, _ = run_gpu(inst, variant=1)
    check_fp32(inst, Z, bound_fn=tc_elem_bound)


# ------------------------------------------------------------------ sparse
def sparse_elem_bound(inst, rows=None):
    """Few terms per element: each FMA rounds once in FP32 (summation in a
    fixed k order), at most nnz(row of X) additions."""
    return (np.count_nonzero(inst.X, axis=1).max(initial=0) + 2) * U32 * \
        abs_product(inst, rows) + 1e-30


@pytest.mark.parametrize("n", [1, 7, 64, 129, 257, 1000])
@pytest.mark.parametrize("case", ["A", "B"])
def test_sparse_quadratic_regime(case, n):
    inst = W.make("caseB_n4096_sparse", n=n, seed=n + 11)
    if case == "A":                    # real X, Rep-factor Y (roles swapped)
        inst = W.Instance("A", inst.Y.T.copy(), inst.X.T.copy(), name="spA",
                          x_dtype="f32", y_dtype="i32", z_dtype="f32",
                          target="fp32")
    Z, info = run_gpu(inst, variant=6)
    assert info["variant"] == 6
    check_fp32(inst, Z, bound_fn=sparse_elem_bound)


def test_sparse_full_size_planner_choice():
    inst = W.make("caseB_n4096_sparse")
    Z, info = run_gpu(inst)            # hints d1 d2 n = 1: the sparse form
    assert info["variant"] == 6
    check_fp32(inst, Z, sample_rows(inst.n, 40), bound_fn=sparse_elem_bound)


def test_sparse_wide_rows_in_column_chunks():
    inst = W.make("caseB_n4096_sparse", n=7000, seed=3)
    Z, _ = run_gpu(inst, variant=6)
    check_fp32(inst, Z, sample_rows(inst.n, 16), bound_fn=sparse_elem_bound)


def test_sparse_more_nonzeros_than_planned_is_reported():
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    n = 300
    rng = np.random.default_rng(12)
    X = torch_of(rng.integers(0, 5, size=(n, n)).astype(np.int32))   # dense
    Y = torch_of(rng.standard_normal((n, n)).astype(np.float32))
    Z = torch.empty((n, n), dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "B", "i32", "f32", "f32", "fp32", variant=6,
                       d1=0.001, d2=0.001))
    p(X, Y, Z)
    with pytest.raises(AfmmError) as e:
        p.sync()
    assert e.value.status == 4          # AFMM_ERR_OVERFLOW_RISK


def _sparse_storage(vals, dt):
    """Device tensor of `vals` stored as dtype `dt`, and the stored values
    read back in FP64 (what the oracle multiplies)."""
    tt = {"u8": torch.uint8, "i8": torch.int8, "i32": torch.int32,
          "f32": torch.float32, "f64": torch.float64}
    if dt in tt:
        t = torch.from_numpy(np.ascontiguousarray(vals)).to(tt[dt])
        back = t.to(torch.float64)
    elif dt == "bf16":
        t = torch.from_numpy(np.ascontiguousarray(vals, np.float32)).to(torch.bfloat16)
        back = t.to(torch.float64)
    else:                                           # e4m3 bytes
        f8 = torch.from_numpy(np.ascontiguousarray(vals, np.float32)).to(torch.float8_e4m3fn)
        back = f8.to(torch.float64)
        t = f8.view(torch.uint8)
    return t.cuda(), back.numpy()


@pytest.mark.parametrize("n", [512, 333])
@pytest.mark.parametrize("xd,yd", [("u8", "f32"), ("i8", "bf16"), ("i32", "f64"),
                                   ("e4m3", "f32")])
def test_sparse_storage_dtypes(xd, yd, n):
    """Every element size through the compaction: n = 512 takes the 16-byte
    load path for all of them, n = 333 the per-element path."""
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for
    rng = np.random.default_rng(n + len(xd + yd))
    d = 3.0 / np.sqrt(n)
    Xi = rng.integers(1, 16, size=(n, n)) * (rng.random((n, n)) < d)
    Yr = rng.standard_normal((n, n)) * (rng.random((n, n)) < d)
    Xt, Xv = _sparse_storage(Xi, xd)
    Yt, Yv = _sparse_storage(Yr, yd)
    inst = W.Instance("B", Xv.astype(np.int64), Yv, x_dtype=xd, y_dtype=yd,
                      z_dtype="f32", target="fp32")
    Z = torch.full((n, n), float("nan"), device="cuda")
    p = Plan(desc_for(inst, variant=6))
    p(Xt, Yt, Z)
    p.sync()
    check_fp32(inst, Z.cpu().numpy(), bound_fn=sparse_elem_bound)


@pytest.mark.parametrize("ldx,ldy,ldz", [(256 + 16, 256 + 4, 256 + 4),   # aligned rows
                                         (256 + 3, 256 + 1, 256 + 5)])   # unaligned
def test_sparse_leading_dimensions(ldx, ldy, ldz):
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(ldx)
    n = 256
    Xb = (rng.integers(1, 9, size=(n, ldx)) * (rng.random((n, ldx)) < 0.06)).astype(np.uint8)
    Yb = (rng.standard_normal((n, ldy)) * (rng.random((n, ldy)) < 0.06)).astype(np.float32)
    Zb = torch.full((n, ldz), 7.0, dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "B", "u8", "f32", "f32", "fp32", variant=6,
                       ldx=ldx, ldy=ldy, ldz=ldz))
    p(torch_of(Xb), torch_of(Yb), Zb)
    p.sync()
    Z = Zb.cpu().numpy()
    inst = W.Instance("B", Xb[:, :n].astype(np.int64), Yb[:, :n], x_dtype="u8",
                      y_dtype="f32")
    check_fp32(inst, Z[:, :n], bound_fn=sparse_elem_bound)
    assert np.all(Z[:, n:] == 7.0)      # padding columns untouched


def test_sparse_one_dense_factor_and_repeat_calls():
    """d1 = 1 with d2 = 2/n (d1 d2 n = 2): a dense Rep-factor matrix is
    compacted too.  A second call gives the same bits (fixed order)."""
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for
    rng = np.random.default_rng(77)
    n = 640
    X = rng.integers(1, 16, size=(n, n)).astype(np.int32)
    Y = (rng.standard_normal((n, n)) * (rng.random((n, n)) < 2.0 / n)).astype(np.float32)
    inst = W.Instance("B", X, Y, x_dtype="i32", y_dtype="f32")
    p = Plan(desc_for(inst))
    assert p.info["variant"] == 6
    Xt, Yt = torch_of(X), torch_of(Y)
    Z1 = torch.full((n, n), float("nan"), device="cuda")
    Z2 = torch.full((n, n), float("nan"), device="cuda")
    p(Xt, Yt, Z1)
    p(Xt, Yt, Z2)
    p.sync()
    check_fp32(inst, Z1.cpu().numpy(), bound_fn=sparse_elem_bound)
    assert torch.equal(Z1, Z2)


def test_sparse_uneven_rows_use_the_overflow_region():
    """A few dense rows among sparse ones: those rows exceed their slot and
    are compacted into the overflow region.  Repeat calls agree bit for bit;
    a call that overflows the region reports it and the next call works."""
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    rng = np.random.default_rng(91)
    n = 512
    X = (rng.integers(1, 16, size=(n, n)) * (rng.random((n, n)) < 1.0 / 16)).astype(np.int32)
    X[[3, 100, 257, 400, 511]] = rng.integers(1, 16, size=(5, n))
    Y = (rng.standard_normal((n, n)) * (rng.random((n, n)) < 1.0 / 16)).astype(np.float32)
    Y[[0, 7]] = rng.standard_normal((2, n))
    inst = W.Instance("B", X, Y, x_dtype="i32", y_dtype="f32")
    d1 = np.count_nonzero(X) / n / n
    d2 = np.count_nonzero(Y) / n / n
    p = Plan(make_desc(n, "B", "i32", "f32", "f32", "fp32", variant=6, d1=d1, d2=d2))
    Xt, Yt = torch_of(X), torch_of(Y)
    Z1 = torch.full((n, n), float("nan"), device="cuda")
    Z2 = torch.full((n, n), float("nan"), device="cuda")
    p(Xt, Yt, Z1)
    p(Xt, Yt, Z2)
    p.sync()
    check_fp32(inst, Z1.cpu().numpy(), bound_fn=sparse_elem_bound)
    assert torch.equal(Z1, Z2)
    # Far more dense rows than the overflow region holds: reported.
    Xd = X.copy()
    Xd[::2] = rng.integers(1, 16, size=(n // 2, n))
    p(torch_of(Xd), Yt, Z2)
    with pytest.raises(AfmmError) as e:
        p.sync()
    assert e.value.status == 4          # AFMM_ERR_OVERFLOW_RISK
    Z3 = torch.full((n, n), float("nan"), device="cuda")
    p(Xt, Yt, Z3)
    p.sync()
    assert torch.equal(Z1, Z3)


# ------------------------------------------------------------------ exact, TC
def exact_case(case, n, seed):
    inst = W.make("caseA_n16384_i8", n=n, seed=seed)
    if case == "B":   # X Rep-factors, Y integer Base values
        inst = W.Instance("B", inst.Y.copy(), inst.X.copy(), name="exactB",
                          x_dtype="i8", y_dtype="i8", z_dtype="i32",
                          target="exact")
    return inst


@pytest.mark.parametrize("n", TC_RAGGED)
@pytest.mark.parametrize("case", ["A", "B"])
def test_tc_exact_ragged(case, n):
    """No magnitude hints: K chunks sized from the int8 bounds (992)."""
    inst = exact_case(case, n, seed=n + 7)
    Z, info = run_gpu(inst, variant=5)
    assert info["variant"] == 5 and info["k_split"] == -(-n // 992)
    assert np.array_equal(Z.astype(np.int64), oracle_rows(inst))


def test_tc_exact_worst_case_magnitudes():
    n = 2048                            # two K chunks at the int8 bounds
    X = np.full((n, n), -128, dtype=np.int8)
    X[1::2] = 127
    Y = np.full((n, n), 127, dtype=np.int8)
    inst = W.Instance("A", X, Y, name="worst", x_dtype="i8", y_dtype="i8",
                      z_dtype="i32", target="exact")
    Z, info = run_gpu(inst, variant=5)
    assert info["k_split"] == 3
    assert np.array_equal(Z.astype(np.int64), oracle_rows(inst))


def test_tc_exact_full_size_sampled_with_hints():
    """n = 16384 with the workload's magnitudes as hints: 2 K chunks."""
    import torch as T
    from paper_1308_2400_gb300 import Plan, make_desc
    inst = W.make("caseA_n16384_i8")
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Z = T.empty((inst.n, inst.n), dtype=T.int32, device="cuda")
    p = Plan(make_desc(inst.n, "A", "i8", "i8", "i32", "exact", variant=5,
                       rep_max=15, base_max=127))
    assert p.info["variant"] == 5 and p.info["k_split"] == 2
    p(X, Y, Z)
    p.sync()
    rows = sample_rows(inst.n, 6)
    assert np.array_equal(Z.cpu().numpy()[rows].astype(np.int64),
                          oracle_rows(inst, rows))


def test_tc_exact_hint_violation_is_reported():
    import torch as T
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    n = 256
    X = T.ones((n, n), dtype=T.int8, device="cuda")
    Y = T.ones((n, n), dtype=T.int8, device="cuda")
    Y[3, 4] = 100                       # above the rep_max hint of 15
    Z = T.empty((n, n), dtype=T.int32, device="cuda")
    p = Plan(make_desc(n, "A", "i8", "i8", "i32", "exact", variant=5,
                       rep_max=15, base_max=127))
    p(X, Y, Z)
    with pytest.raises(AfmmError) as e:
        p.sync()
    assert e.value.status == 4          # AFMM_ERR_OVERFLOW_RISK


# ------------------------------------------------- exact, TC, E4M3 digits
X8 = 11                        # AFMM_VARIANT_TC_EXACT_F8


@pytest.mark.parametrize("n", [512, 513, 600, 1000, 1537])
@pytest.mark.parametrize("case", ["A", "B"])
def test_tc_exact_f8_ragged(case, n):
    """Two E4M3 digits of the integer Base factor, CTA pairs, int32
    epilogue (Case B: tiles of Z^T stored transposed): bit-exact."""
    inst = exact_case(case, n, seed=n + 3)
    Z, info = run_gpu(inst, variant=X8)
    assert info["variant"] == X8
    assert np.array_equal(Z.astype(np.int64), oracle_rows(inst))


@pytest.mark.parametrize("xd,n,pad", [("u8", 512, 0), ("i8", 520, 0), ("u8", 600, 8),
                                      ("i8", 777, 0), ("u8", 513, 3)])
def test_tc_exact_f8_one_byte_base_values_every_code(xd, n, pad):
    """int8 and uint8 Base values: their digits are the two nibbles, coded
    by table when rows are 8-byte aligned (n + pad a multiple of 8) and by
    the per-element path otherwise; every byte value appears in every
    column position of the first 256 rows; uint8 Rep-factors.  Bit-exact."""
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(n + pad)
    lo = 0 if xd == "u8" else -128
    X = rng.integers(lo, lo + 256, size=(n, n))
    r = np.arange(256).reshape(-1, 1)
    X[:256] = (r + np.arange(n).reshape(1, -1)) % 256 + lo
    Y = rng.integers(0, 17, size=(n, n))
    ld = n + pad
    npdt = np.uint8 if xd == "u8" else np.int8
    Xb = np.zeros((n, ld), dtype=npdt)
    Xb[:, :n] = X
    Z = torch.full((n, n), -7, dtype=torch.int32, device="cuda")
    p = Plan(make_desc(n, "A", xd, "u8", "i32", "exact", variant=X8, ldx=ld))
    p(torch_of(Xb), torch_of(Y.astype(np.uint8)), Z)
    p.sync()
    p.close()
    inst = W.Instance("A", X, Y, name=f"bytes_{xd}", x_dtype=xd, y_dtype="u8",
                      z_dtype="i32", target="exact")
    assert np.array_equal(Z.cpu().numpy().astype(np.int64), oracle_rows(inst))


def test_tc_exact_f8_worst_case_digits():
    """Base values at +-255 and at digit boundaries (-1, -16, 15, 16),
    Rep-factors at 16: the largest digit sums the form allows."""
    n = 1024
    X = np.full((n, n), -255, dtype=np.int32)
    X[1::2] = 255
    X[::3, ::5] = -1
    X[::7, ::2] = -16
    X[::5, 1::3] = 15
    X[::11, ::7] = 16
    Y = np.full((n, n), 16, dtype=np.int32)
    Y[::4] = 0
    inst = W.Instance("A", X, Y, name="worst_digits", x_dtype="i32", y_dtype="i32",
                      z_dtype="i32", target="exact")
    Z, _ = run_gpu(inst, variant=X8)
    assert np.array_equal(Z.astype(np.int64), oracle_rows(inst))


def test_tc_exact_f8_full_size_sampled_auto():
    """n = 16384 with the workload's magnitudes as hints: the planner takes
    the E4M3 digit form."""
    import torch as T
    from paper_1308_2400_gb300 import Plan, make_desc
    inst = W.make("caseA_n16384_i8")
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Z = T.empty((inst.n, inst.n), dtype=T.int32, device="cuda")
    p = Plan(make_desc(inst.n, "A", "i8", "i8", "i32", "exact", rep_max=15, base_max=127))
    assert p.info["variant"] == X8
    p(X, Y, Z)
    p.sync()
    p.close()
    rows = sample_rows(inst.n, 6)
    assert np.array_equal(Z.cpu().numpy()[rows].astype(np.int64), oracle_rows(inst, rows))


@pytest.mark.parametrize("where,value,code", [("X", 256, 4), ("Y", 17, 4), ("Y", -1, 3)])
def test_tc_exact_f8_range_errors(where, value, code):
    """A Base value past 255 or a Rep-factor past 16 is AFMM_ERR_OVERFLOW_RISK,
    a negative Rep-factor AFMM_ERR_NEGATIVE_REP."""
    import torch as T
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    n = 600
    X = T.ones((n, n), dtype=T.int32, device="cuda")
    Y = T.ones((n, n), dtype=T.int32, device="cuda")
    (X if where == "X" else Y)[3, 4] = value
    Z = T.empty((n, n), dtype=T.int32, device="cuda")
    p = Plan(make_desc(n, "A", "i32", "i32", "i32", "exact", variant=X8))
    p(X, Y, Z)
    with pytest.raises(AfmmError) as e:
        p.sync()
    assert e.value.status == code
    p.close()


def test_tc_exact_f8_refuses_small():
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    for case in ("A", "B"):
        with pytest.raises(AfmmError) as e:
            Plan(make_desc(256, case, "i8", "i8", "i32", "exact", variant=X8))
        assert e.value.status == 2      # AFMM_ERR_UNSUPPORTED


# ------------------------------------------------------------------ exact
@pytest.mark.parametrize("n", RAGGED)
@pytest.mark.parametrize("case", ["A", "B"])
def test_simt_exact_ragged(case, n):
    inst = W.make("caseA_n16384_i8", n=n, seed=n)
    if case == "B":   # X Rep-factors, Y integer Base values
        inst = W.Instance("B", inst.Y.copy(), inst.X.copy(), name="exactB",
                          x_dtype="i8", y_dtype="i8", z_dtype="i32",
                          target="exact")
    Z, info = run_gpu(inst, variant=4)
    R = oracle_rows(inst)
    assert np.array_equal(Z.astype(np.int64), R)


def test_simt_exact_worst_case_magnitudes():
    """All entries at the int8 extremes: |Z| reaches n * 128 * 127."""
    n = 1024
    X = np.full((n, n), -128, dtype=np.int8)
    X[1::2] = 127
    Y = np.full((n, n), 127, dtype=np.int8)
    inst = W.Instance("A", X, Y, name="worst", x_dtype="i8", y_dtype="i8",
                      z_dtype="i32", target="exact")
    Z, _ = run_gpu(inst, variant=4)
    assert np.array_equal(Z.astype(np.int64), oracle_rows(inst))


def test_simt_exact_full_size_sampled():
    inst = W.make("caseA_n16384_i8")
    Z, _ = run_gpu(inst, variant=4)
    rows = sample_rows(inst.n, 6)
    assert np.array_equal(Z[rows].astype(np.int64), oracle_rows(inst, rows))


# ------------------------------------------------------------------ FP64
def f64slice_elem_bound(inst):
    """Truncation of 56-bit row-scaled digits (< 2^(E_i - 56) per entry,
    E_i the row's exponent bound <= 2 max|x|) plus the FP64 recombination
    (9 roundings of at most 2 sum|x y| each)."""
    real = inst.X if inst.case == "A" else inst.Y.T
    rep = inst.Y if inst.case == "A" else inst.X.T
    rowmax = np.abs(real.astype(np.float64)).max(axis=1, initial=0.0)
    trunc = (2.0 * rowmax * 2.0 ** -56)[:, None] * np.abs(rep).sum(axis=0)[None, :]
    if inst.case == "B":
        trunc = trunc.T
    return trunc + 24 * U64 * abs_product(inst) + 1e-300


@pytest.mark.parametrize("n", RAGGED + [256])
@pytest.mark.parametrize("case", ["A", "B"])
def test_simt_f64slice(case, n):
    inst = W.make("caseA_n256_f64", n=n, seed=n)
    if case == "B":
        inst = W.Instance("B", inst.Y.copy(), inst.X.T.copy(), name="f64B",
                          x_dtype="i32", y_dtype="f64", z_dtype="f64",
                          target="fp64")
    Z, info = run_gpu(inst, variant=3)
    R = oracle_rows(inst)
    assert rel_fro(Z, R) <= FP64_REL_FRO
    assert not (np.abs(Z - R) > f64slice_elem_bound(inst)).any()


def test_simt_f64slice_config_size():
    inst = W.make("caseA_n256_f64")
    Z, info = run_gpu(inst)               # planner picks the FP64 form
    assert info["variant"] == 3 and info["slices"] == 8
    R = oracle_rows(inst)
    assert rel_fro(Z, R) <= FP64_REL_FRO


def test_f64slice_wide_dynamic_range():
    """Rows mixing magnitudes 2^-40 .. 2^40: row scaling keeps 1e-12."""
    rng = np.random.default_rng(5)
    n = 96
    X = rng.uniform(-1, 1, size=(n, n)) * 2.0 ** rng.integers(-40, 41, size=(n, 1))
    Y = rng.integers(0, 10, size=(n, n)).astype(np.int32)
    inst = W.Instance("A", X, Y, name="range", x_dtype="f64", y_dtype="i32",
                      z_dtype="f64", target="fp64")
    Z, _ = run_gpu(inst, variant=3)
    R = oracle_rows(inst)
    rel_rows = np.linalg.norm(Z - R, axis=1) / np.maximum(np.linalg.norm(R, axis=1), 1e-300)
    assert rel_rows.max() <= FP64_REL_FRO


# ------------------------------------------------------------------ boundary
def test_validation_reports_bad_rep_factors():
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    n = 70
    X = torch.ones((n, n), dtype=torch.float32, device="cuda")
    Y = torch.ones((n, n), dtype=torch.int32, device="cuda")
    Y[5, 7] = -2
    Z = torch.empty((n, n), dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "A", "f32", "i32", "f32", "fp32", variant=0,
                       flags=1))
    p(X, Y, Z)
    with pytest.raises(AfmmError) as e:
        p.sync()
    assert e.value.status == 3          # AFMM_ERR_NEGATIVE_REP
    Yf = torch.ones((n, n), dtype=torch.float32, device="cuda")
    Yf[0, 0] = 0.5
    q = Plan(make_desc(n, "A", "f32", "f32", "f32", "fp32", variant=0,
                       flags=1))
    q(X, Yf, Z)
    with pytest.raises(AfmmError) as e:
        q.sync()
    assert e.value.status == 9          # AFMM_ERR_NONINTEGER_REP
    Y[5, 7] = 3                          # the status word was cleared
    p(X, Y, Z)
    p.sync()


def test_validation_measures_paper_parameters():
    from oracle import expected_additions, realised_parameters
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for
    inst = W.make("caseB_n4096_f32", n=300, seed=9)
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Z = torch.empty((300, 300), dtype=torch.float32, device="cuda")
    p = Plan(desc_for(inst, variant=0, flags=1, hints=False))
    p(X, Y, Z)
    p.sync()
    info = p.info
    ref = realised_parameters(inst.X, inst.Y, "B")
    for k in ("d1", "d2", "mu_prime", "mu"):
        assert abs(info[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    e = expected_additions(ref["mu_prime"], ref["d1"], ref["d2"], 300)
    assert abs(info["expected_additions"] - e) <= 1e-9 * e
    assert info["rep_max"] == inst.X.max()


def test_host_buffers_match_device_buffers():
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for
    inst = W.make("caseB_n4096_f32", n=200, seed=2)
    Zd, _ = run_gpu(inst, variant=0)
    Zh = np.full((200, 200), np.nan, dtype=np.float32)
    p = Plan(desc_for(inst, variant=0))
    p(np.ascontiguousarray(inst.X), np.ascontiguousarray(inst.Y), Zh)
    p.sync()
    assert np.array_equal(Zh, Zd)
    # pinned host memory
    Xp = torch.from_numpy(inst.X).pin_memory()
    Yp = torch.from_numpy(inst.Y).pin_memory()
    Zp = torch.empty((200, 200), dtype=torch.float32).pin_memory()
    p(Xp, Yp, Zp)
    p.sync()
    assert np.array_equal(Zp.numpy(), Zd)


@pytest.mark.parametrize("case", ["A", "B"])
def test_host_buffers_pipelined_tensor_core_path(case):
    """Host X, Y, Z with the split tensor-core form: Y is copied in first,
    then row blocks of X are copied in, multiplied and copied out on three
    streams.  The result is bit-identical to the device-resident call."""
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for
    wl = "caseA_n8192_e4m3" if case == "A" else "caseB_n4096_f32"
    inst = W.make(wl, n=1500, seed=21)
    Zd, _ = run_gpu(inst, variant=1)
    Xs = inst.x_store if inst.x_store is not None else inst.X
    Ys = inst.y_store if inst.y_store is not None else inst.Y
    p = Plan(desc_for(inst, variant=1))
    for pinned in (False, True):
        Xh = torch.from_numpy(np.ascontiguousarray(Xs))
        Yh = torch.from_numpy(np.ascontiguousarray(Ys))
        Zh = torch.full((inst.n, inst.n), float("nan"))
        if pinned:
            Xh, Yh, Zh = Xh.pin_memory(), Yh.pin_memory(), Zh.pin_memory()
        p(Xh, Yh, Zh)
        p.sync()
        assert np.array_equal(Zh.numpy(), Zd), (case, pinned)


@pytest.mark.parametrize("variant", [0, 1])
def test_leading_dimensions(variant):
    """Padded rows on all three matrices (ldz = n + 5: rows of Z off 16-byte
    boundaries, which the tensor-core form writes through an aligned buffer
    and a 2-D copy); the padding columns of Z are left alone."""
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(4)
    n, pad = 131, 9
    Xb = rng.uniform(-1, 1, size=(n, n + pad)).astype(np.float32)
    Yb = rng.integers(0, 9, size=(n, n + pad + 3)).astype(np.int32)
    X, Y = Xb[:, :n], Yb[:, :n]
    Zb = torch.full((n, n + 5), 7.0, dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "A", "f32", "i32", "f32", "fp32", variant=variant,
                       ldx=n + pad, ldy=n + pad + 3, ldz=n + 5))
    p(torch_of(Xb), torch_of(Yb), Zb)
    p.sync()
    Z = Zb.cpu().numpy()
    inst = W.Instance("A", X, Y, x_dtype="f32", y_dtype="i32")
    check_fp32(inst, Z[:, :n], bound_fn=tc_elem_bound if variant == 1 else None)
    assert np.all(Z[:, n:] == 7.0)      # padding columns untouched


@pytest.mark.parametrize("workload,variant", [("caseA_n256_f64", -1), ("caseB_n4096_f32", 1),
                                              ("caseB_n4096_sparse", 6)])
def test_repeated_calls_replay_a_graph(workload, variant):
    """From the third call in a row on the same device buffers the product
    is replayed from a CUDA graph.  Replays read the buffers' current
    contents, give the bits of an eager call, and count their launches;
    new buffers start over."""
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for, gpu_operands, z_torch_dtype
    inst = W.make(workload, n=300, seed=5)
    inst2 = W.make(workload, n=300, seed=6)
    p = Plan(desc_for(inst, variant=variant))
    X, Y = gpu_operands(inst)
    X2, Y2 = gpu_operands(inst2)
    zt = z_torch_dtype(inst.z_dtype)
    Z = torch.empty((300, 300), dtype=zt, device="cuda")
    outs = []
    for _ in range(5):
        p(X, Y, Z)
        p.sync()
        outs.append(Z.clone())
    c = p.counters()
    assert c["calls"] == 5 and c["kernel_launches"] % 5 == 0
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    def check(ins, Zn):
        if ins.target == "fp64":
            assert rel_fro(Zn, oracle_rows(ins)) <= FP64_REL_FRO
        else:
            check_fp32(ins, Zn, bound_fn=sparse_elem_bound if variant == 6 else tc_elem_bound)

    check(inst, outs[0].cpu().numpy())
    # New contents in the same buffers: the replay reads them.
    X.copy_(X2)
    Y.copy_(Y2)
    p(X, Y, Z)
    p.sync()
    check(inst2, Z.cpu().numpy())
    # Other buffers: eager again, then a new capture.
    Z2 = torch.empty_like(Z)
    for _ in range(4):
        p(X2, Y2, Z2)
    p.sync()
    assert torch.equal(Z2, Z)


def test_empty_problem():
    from paper_1308_2400_gb300 import Plan, make_desc
    p = Plan(make_desc(0, "A", "f32", "i32", "f32", "fp32"))
    e = torch.empty((0, 0), dtype=torch.float32, device="cuda")
    p(e, torch.empty((0, 0), dtype=torch.int32, device="cuda"), e)
    p.sync()


def test_error_norm_kernel():
    from paper_1308_2400_gb300 import afmm_error_norm
    rng = np.random.default_rng(6)
    R = rng.standard_normal((333, 517))
    Z = (R + 1e-7 * rng.standard_normal(R.shape)).astype(np.float32)
    d, r, m = afmm_error_norm(torch_of(Z), "f32", 517, torch_of(R), "f64",
                              517, 333, 517)
    D = Z.astype(np.float64) - R
    assert abs(d - np.linalg.norm(D)) <= 1e-12 * np.linalg.norm(D)
    assert abs(r - np.linalg.norm(R)) <= 1e-12 * np.linalg.norm(R)
    assert m == np.abs(D).max()


def _batch(insts, routes=None):
    """Device operands, descriptors (forced route when given) and outputs."""
    from _helpers import desc_for, gpu_operands
    descs, Xs, Ys, Zs = [], [], [], []
    for t, inst in enumerate(insts):
        X, Y = gpu_operands(inst)
        v = -1 if routes is None else routes[t]
        descs.append(desc_for(inst, variant=v))
        Xs.append(X)
        Ys.append(Y)
        Zs.append(torch.full((inst.n, inst.n), float("nan"), dtype=torch.float32,
                             device="cuda"))
    return descs, Xs, Ys, Zs


def _check_batch(insts, Zs, descs=None, rows_per_instance=None):
    """Every instance against the oracle: relative Frobenius error and the
    element bound of the route it took (tensor cores or CUDA cores; the
    route read back from the dispatcher when descriptors are given), on
    all rows or on a sampled set per instance."""
    from paper_1308_2400_gb300 import afmm as A
    for t, (inst, Z) in enumerate(zip(insts, Zs)):
        rows = None if rows_per_instance is None else \
            sample_rows(inst.n, rows_per_instance, seed=t)
        R = oracle_rows(inst, rows)
        Zn = Z.cpu().numpy()
        Zn = Zn if rows is None else Zn[rows]
        assert np.all(np.isfinite(Zn)), inst.name
        assert rel_fro(Zn, R) <= FP32_REL_FRO, inst.name
        if descs is not None:
            tc = A.afmm_dispatch_variant(descs[t]) in (A.AFMM_VARIANT_TC_BF16X3,
                                                       A.AFMM_VARIANT_TC_BF16X3_N128)
            bound = (tc_elem_bound if tc else simt_f32_elem_bound)(inst, rows)
            bad = np.abs(Zn.astype(np.float64) - R) > bound
            assert not bad.any(), (inst.name, "tc" if tc else "simt", int(bad.sum()))


@pytest.mark.parametrize("route", ["auto", "tc", "tc128", "simt", "mixed"])
def test_batched_grouped_routes(route):
    """Every route of the batched call, alone and mixed in one batch: the
    CUDA-core form (variant 0), tensor cores with 128 x 256 tiles (1) and
    with 128 x 128 tiles (9), both tile widths sharing one grouped launch."""
    from paper_1308_2400_gb300 import afmm_mul_batched
    from paper_1308_2400_gb300.afmm import afmm_batched_sync
    insts = W.batched_mix(count=14, seed=5, n_min=16, n_max=400)
    routes = {"auto": None, "tc": [1] * 14, "tc128": [9] * 14, "simt": [0] * 14,
              "mixed": [(0, 1, 9)[t % 3] for t in range(14)]}[route]
    descs, Xs, Ys, Zs = _batch(insts, routes)
    afmm_mul_batched(descs, Xs, Ys, Zs)
    afmm_batched_sync(descs)
    _check_batch(insts, Zs, descs=descs)


def test_batched_graph_replay_with_new_data():
    """Same descriptors, new operands: the cached plan and graph must read
    the new pointers."""
    from paper_1308_2400_gb300 import afmm_mul_batched
    from paper_1308_2400_gb300.afmm import afmm_batched_sync
    first = W.batched_mix(count=9, seed=6, n_min=40, n_max=300)
    descs, Xs, Ys, Zs = _batch(first, [t % 2 for t in range(9)])
    afmm_mul_batched(descs, Xs, Ys, Zs)
    afmm_batched_sync(descs)
    _check_batch(first, Zs)
    second = W.batched_mix(count=9, seed=6, n_min=40, n_max=300)
    rng = np.random.default_rng(7)
    for inst in second:                 # same shapes and kinds, new values
        real = inst.X if inst.case == "A" else inst.Y
        real *= rng.uniform(0.5, 2.0, size=real.shape).astype(real.dtype)
    _, Xs2, Ys2, Zs2 = _batch(second, [t % 2 for t in range(9)])
    afmm_mul_batched(descs, Xs2, Ys2, Zs2)
    afmm_batched_sync(descs)
    _check_batch(second, Zs2)


def test_batched_bad_rep_factor_poisons_only_its_instance():
    """A Rep-factor not exact in BF16 (300) on the tensor-core route turns
    that instance's Z into NaN and is reported by afmm_batched_sync; the
    other instance is unaffected."""
    from paper_1308_2400_gb300 import AfmmError, afmm_mul_batched
    from paper_1308_2400_gb300.afmm import AFMM_ERR_OVERFLOW_RISK, afmm_batched_sync
    rng = np.random.default_rng(9)
    insts = []
    for t in range(2):
        n = 150 + 20 * t
        X = rng.standard_normal((n, n)).astype(np.float32)
        Y = rng.integers(0, 9, size=(n, n)).astype(np.int32)
        insts.append(W.Instance("A", X, Y, name=f"b{t}", x_dtype="f32",
                                y_dtype="i32", z_dtype="f32", target="fp32"))
    insts[0].Y[3, 5] = 300
    descs, Xs, Ys, Zs = _batch(insts, [1, 1])
    afmm_mul_batched(descs, Xs, Ys, Zs)
    with pytest.raises(AfmmError) as e:
        afmm_batched_sync(descs)
    assert e.value.status == AFMM_ERR_OVERFLOW_RISK
    assert np.all(np.isnan(Zs[0].cpu().numpy()))
    _check_batch(insts[1:], Zs[1:])


def test_batched_law_with_learned_dispatch():
    """The batched workload's own law (n log-uniform up to 2048, d1, d2 in
    [0.05, 1], Poisson Rep-factors, cases A and B) at 64 instances, routed
    by the installed dispatch network: every instance checked against the
    oracle on sampled rows, with the element bound of its route."""
    from paper_1308_2400_gb300 import afmm_mul_batched
    from paper_1308_2400_gb300 import tune
    from paper_1308_2400_gb300.afmm import afmm_batched_sync, afmm_set_dispatch_model
    insts = W.batched_mix(count=64, seed=17)
    assert max(t.n for t in insts) > 1024 and {t.case for t in insts} == {"A", "B"}
    tune.install(tune.load(tune.DEFAULT_MODEL))
    try:
        descs, Xs, Ys, Zs = _batch(insts)
        afmm_mul_batched(descs, Xs, Ys, Zs)
        afmm_batched_sync(descs)
        _check_batch(insts, Zs, descs=descs, rows_per_instance=10)
    finally:
        afmm_set_dispatch_model(None, None, None, None, None)


def test_batched_small_mix():
    from paper_1308_2400_gb300 import afmm_mul_batched
    insts = W.batched_mix(count=10, seed=1, n_min=16, n_max=160)
    descs, Xs, Ys, Zs = _batch(insts)
    afmm_mul_batched(descs, Xs, Ys, Zs)
    torch.cuda.synchronize()
    _check_batch(insts, Zs)


_DEGENERATE_FORMS = {   # variant: (X dtype, Y dtype, Z dtype, target)
    0: ("f32", "i32", "f32", "fp32"), 1: ("f32", "i32", "f32", "fp32"),
    6: ("f32", "i32", "f32", "fp32"), 3: ("f64", "i32", "f64", "fp64"),
    4: ("i8", "i8", "i32", "exact"), 5: ("i8", "i8", "i32", "exact"),
    7: ("f32", "i32", "f32", "fp32"),
}


@pytest.mark.parametrize("kind", ["zero_base", "zero_rep", "unit_rep"])
@pytest.mark.parametrize("variant", sorted(_DEGENERATE_FORMS))
def test_degenerate_inputs(variant, kind):
    """The method's degenerate cases on every form: no non-zero Base
    (Z = 0, no additions), no non-zero Rep-factor (Z = 0), and every
    Rep-factor 1 (each Z[i,j] is a row sum of the Base values)."""
    xd, yd, zd, target = _DEGENERATE_FORMS[variant]
    rng = np.random.default_rng(variant * 7 + len(kind))
    n = 200
    if xd == "i8":
        X = rng.integers(-127, 128, size=(n, n)).astype(np.int8)
    else:
        X = rng.uniform(-1, 1, size=(n, n)).astype(np.float32 if xd == "f32" else np.float64)
    Y = rng.integers(0, 9, size=(n, n)).astype(np.int8 if yd == "i8" else np.int32)
    if kind == "zero_base":
        X[:] = 0
    elif kind == "zero_rep":
        Y[:] = 0
    else:
        Y[:] = 1
    inst = W.Instance("A", X, Y, x_dtype=xd, y_dtype=yd, z_dtype=zd, target=target)
    Z, info = run_gpu(inst, variant=variant)
    assert info["variant"] == variant
    if kind != "unit_rep":
        assert np.all(Z == 0), kind
        return
    R = oracle_rows(inst)
    if target == "exact":
        assert np.array_equal(Z.astype(np.int64), R)
    elif target == "fp64":
        assert rel_fro(Z, R) <= FP64_REL_FRO
    else:
        assert rel_fro(Z, R) <= FP32_REL_FRO


# ------------------------------------------------------- K0 tile masks (K1)
def _expected_k_tiles(A, B):
    """k tiles the zero-skip kernel multiplies: per 64 x 256 output tile,
    the 32-wide k tiles whose 64 x 32 tile of A and 32 x 256 tile of B both
    hold a non-zero (counted here from the data, in numpy)."""
    n = A.shape[0]
    mb, kb, nb = -(-n // 64), -(-n // 32), -(-n // 256)
    xm = np.zeros((mb, kb), bool)
    ym = np.zeros((kb, nb), bool)
    for i in range(mb):
        for t in range(kb):
            xm[i, t] = np.any(A[i * 64:(i + 1) * 64, t * 32:(t + 1) * 32] != 0)
    for t in range(kb):
        for j in range(nb):
            ym[t, j] = np.any(B[t * 32:(t + 1) * 32, j * 256:(j + 1) * 256] != 0)
    return int((xm.astype(np.int64) @ ym.astype(np.int64)).sum())


@pytest.mark.parametrize("case", ["A", "B"])
def test_simt_tile_masks_skip_zero_blocks(case):
    """Zero bands and blocks in both factors: the zero-skip kernel multiplies
    exactly the k tiles the masks leave live, and Z matches the oracle."""
    from paper_1308_2400_gb300 import Plan
    rng = np.random.default_rng(21 if case == "A" else 22)
    n = 515
    real = rng.uniform(-1, 1, size=(n, n)).astype(np.float32)
    real[rng.random((n, n)) > 0.3] = 0
    rep = rng.poisson(3.0, size=(n, n)).astype(np.int32)
    if case == "A":
        X, Y = real, rep
    else:
        X, Y = rep, real
    X[:, 64:160] = 0                    # k tiles 2..4 of every row block
    X[128:256, :] = 0                   # row blocks 2 and 3
    Y[320:352, 0:256] = 0               # k tile 10 of column block 0
    Y[480:, 256:512] = 0                # k tiles 15, 16 of column block 1
    inst = W.Instance(case, X, Y, name="blocks" + case, x_dtype="f32" if case == "A" else "i32",
                      y_dtype="i32" if case == "A" else "f32", z_dtype="f32",
                      target="fp32")
    Xg, Yg = torch_of(X), torch_of(Y)
    Z = torch.full((n, n), float("nan"), device="cuda")
    plan = Plan(desc_for(inst, variant=0, d1_hint=0.05))
    plan(Xg, Yg, Z)
    plan.sync()
    got = plan.counters()["simt_k_tiles"]
    plan(Xg, Yg, Z)
    plan.sync()
    again = plan.counters()["simt_k_tiles"]
    plan.close()
    want = _expected_k_tiles(X.astype(np.float32), Y.astype(np.float32))
    assert want < -(-n // 64) * -(-n // 256) * -(-n // 32)     # some tiles skipped
    assert got == want and again == 2 * want
    Zn = Z.cpu().numpy()
    check_fp32(inst, Zn)
    assert np.all(Zn[128:256] == 0)


def test_simt_dense_kernel_reports_no_k_tiles():
    from paper_1308_2400_gb300 import Plan
    inst = W.make("caseA_n8192_e4m3", n=130, seed=4)
    plan = Plan(desc_for(inst, variant=0))
    X, Y = gpu_operands(inst)
    Z = torch.empty((inst.n, inst.n), device="cuda")
    plan(X, Y, Z)
    plan.sync()
    assert plan.counters()["simt_k_tiles"] == -1
    plan.close()


# ------------------------------------------------------ FP16 two-slice form
F16X2 = 10                      # AFMM_VARIANT_TC_F16X2
F16_RAGGED = [1, 7, 33, 127, 129, 255, 257, 300, 513, 600]


@pytest.mark.parametrize("n", F16_RAGGED)
def test_tc_f16x2_ragged(n):
    """Two FP16 slices, one-CTA kernel below n = 512, CTA pairs from it."""
    inst = W.make("caseA_n8192_e4m3", n=n, seed=n + 7)
    Z, info = run_gpu(inst, variant=F16X2)
    assert info["variant"] == F16X2 and info["slices"] == 2
    check_fp32(inst, Z, bound_fn=tc_elem_bound)


def test_tc_f16x2_full_size_sampled():
    inst = W.make("caseA_n8192_e4m3")
    Z, _ = run_gpu(inst, variant=F16X2)
    err = check_fp32(inst, Z, sample_rows(inst.n, 12), bound_fn=tc_elem_bound)
    assert err < 5e-7


def test_tc_f16x2_row_scales():
    """Rows 2^-120 .. 2^100 apart, a zero row and a row of FP32 subnormals:
    each row's own power of two keeps its slices in FP16's range."""
    rng = np.random.default_rng(17)
    n = 300
    X = rng.uniform(-1, 1, size=(n, n))
    X[rng.random((n, n)) > 0.7] = 0
    X *= np.exp2(np.linspace(-120, 100, n)).reshape(n, 1)
    X[5] = 0
    X[6] = rng.uniform(-1, 1, n) * 1e-40
    X = X.astype(np.float32)
    Y = rng.integers(0, 17, size=(n, n)).astype(np.int32)
    inst = W.Instance("A", X, Y, name="scales", x_dtype="f32", y_dtype="i32",
                      z_dtype="f32", target="fp32")
    Z, _ = run_gpu(inst, variant=F16X2)
    check_fp32(inst, Z, bound_fn=tc_elem_bound)
    assert np.all(Z[5] == 0)


def test_tc_f16x2_rep_factor_limit():
    """Rep-factors up to 2048 are exact in FP16; 2049 is refused."""
    from paper_1308_2400_gb300 import AfmmError, Plan
    from paper_1308_2400_gb300.afmm import AFMM_ERR_OVERFLOW_RISK
    rng = np.random.default_rng(5)
    n = 130
    X = rng.uniform(-1, 1, size=(n, n)).astype(np.float32)
    Y = rng.integers(0, 2049, size=(n, n)).astype(np.int32)
    Y[3, 4] = 2048
    inst = W.Instance("A", X, Y, name="big_rep", x_dtype="f32", y_dtype="i32",
                      z_dtype="f32", target="fp32")
    Z, _ = run_gpu(inst, variant=F16X2)
    check_fp32(inst, Z, bound_fn=tc_elem_bound)
    Y[7, 9] = 2049
    Xg, Yg = torch_of(X), torch_of(Y)
    Zg = torch.empty((n, n), device="cuda")
    plan = Plan(desc_for(inst, variant=F16X2))
    plan(Xg, Yg, Zg)
    with pytest.raises(AfmmError) as e:
        plan.sync()
    assert e.value.status == AFMM_ERR_OVERFLOW_RISK
    plan.close()


@pytest.mark.parametrize("n", [1, 33, 129, 300, 513, 600])
def test_tc_f16x2_case_b_ragged(n):
    """Case B as Z^T = Y^T X^T: Y's columns scaled and split, X's
    Rep-factors as FP16 rows; both kernels."""
    inst = W.make("caseB_n4096_f32", n=n, seed=n + 11)
    Z, info = run_gpu(inst, variant=F16X2)
    assert info["variant"] == F16X2
    check_fp32(inst, Z, bound_fn=tc_elem_bound)


def test_tc_f16x2_case_b_full_size_sampled():
    inst = W.make("caseB_n4096_f32")
    Z, _ = run_gpu(inst, variant=F16X2)
    err = check_fp32(inst, Z, sample_rows(inst.n, 16), bound_fn=tc_elem_bound)
    assert err < 5e-7


def test_tc_f16x2_case_b_column_scales():
    """Columns of Y 2^-100 .. 2^100 apart and an all-zero column."""
    rng = np.random.default_rng(19)
    n = 260
    X = rng.integers(0, 16, size=(n, n)).astype(np.int32)
    X[rng.random((n, n)) > 0.5] = 0
    Y = rng.standard_normal((n, n)) * np.exp2(np.linspace(-100, 100, n)).reshape(1, n)
    Y[:, 7] = 0
    Y = Y.astype(np.float32)
    inst = W.Instance("B", X, Y, name="colscales", x_dtype="i32", y_dtype="f32",
                      z_dtype="f32", target="fp32")
    Z, _ = run_gpu(inst, variant=F16X2)
    check_fp32(inst, Z, bound_fn=tc_elem_bound)
    assert np.all(Z[:, 7] == 0)
