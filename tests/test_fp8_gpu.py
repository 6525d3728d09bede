"""Parity of the FP8 (E4M3) tensor-core form with the CPU oracle (GPU tests).

The real factor is cut, row by row (Case A: rows of X; Case B: columns of
Y, the rows of the A operand of Z^T = Y^T X^T), into four E4M3 slices after
a power-of-two scaling that puts the row's largest |value| in [128, 256);
the Rep-factors are held exactly in E4M3.  Per element the slices miss the
value by at most 2^-16 |v| or 2^-21 times the row's largest |value|, so

    |Z - XY|_ij <= sum_k (2^-16 |x_ik| + 2^-21 m_i) y_kj + accumulation

(Case A, m_i = max_k |x_ik|; Case B the same with Y's column maxima), the
accumulation term being that of the BF16 form (FP32 sums in TMEM).  Every
test also holds the 1e-6 relative Frobenius bar of the FP32 target.
"""
from __future__ import annotations

import numpy as np
import pytest

import afmm_inputs as W
from _helpers import (FP32_REL_FRO, U32, abs_product, oracle_rows, rel_fro, run_gpu,
                      sample_rows, torch_of)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP8 = 7
TC_RAGGED = [1, 7, 33, 127, 128, 129, 255, 256, 257, 300, 513]


def fp8_elem_bound(inst, rows=None):
    X = np.abs(inst.X.astype(np.float64))
    Y = np.abs(inst.Y.astype(np.float64))
    acc = 2 * (2 * -(-inst.n // 16) + 8) * U32 * abs_product(inst, rows)
    if inst.case == "A":
        Xr = X if rows is None else X[rows]
        m = Xr.max(axis=1, initial=0.0)[:, None]
        trunc = 2.0 ** -16 * (Xr @ Y) + 2.0 ** -21 * m * Y.sum(axis=0)[None, :]
    else:
        m = Y.max(axis=0, initial=0.0)[None, :]
        Xr = X if rows is None else X[rows]
        trunc = 2.0 ** -16 * (Xr @ Y) + 2.0 ** -21 * Xr.sum(axis=1)[:, None] * m
    return acc + trunc + 1e-30


def check(inst, Z, rows=None):
    R = oracle_rows(inst, rows)
    Zs = Z if rows is None else Z[rows]
    assert np.all(np.isfinite(Zs))
    err = rel_fro(Zs, R)
    assert err <= FP32_REL_FRO, (inst.name, err)
    bad = np.abs(Zs.astype(np.float64) - R) > fp8_elem_bound(inst, rows)
    assert not bad.any(), (inst.name, int(bad.sum()))
    return err


@pytest.mark.parametrize("n", TC_RAGGED)
@pytest.mark.parametrize("workload", ["caseA_n8192_e4m3", "caseB_n4096_f32"])
def test_fp8_ragged(workload, n):
    inst = W.make(workload, n=n, seed=n + 11)
    Z, info = run_gpu(inst, variant=FP8)
    assert info["variant"] == FP8 and info["slices"] == 4
    check(inst, Z)


def test_fp8_case_a_full_size_sampled():
    inst = W.make("caseA_n8192_e4m3")
    Z, _ = run_gpu(inst, variant=FP8)
    check(inst, Z, sample_rows(inst.n, 12))


def test_fp8_case_b_full_size_sampled():
    inst = W.make("caseB_n4096_f32")
    Z, _ = run_gpu(inst, variant=FP8)
    check(inst, Z, sample_rows(inst.n, 24))


def _stored(vals, dt):
    """Device tensor of `vals` stored as dtype `dt` and the stored values in
    FP64 (what the oracle multiplies)."""
    tt = {"u8": torch.uint8, "i8": torch.int8, "i32": torch.int32,
          "f32": torch.float32, "f64": torch.float64}
    if dt in tt:
        t = torch.from_numpy(np.ascontiguousarray(vals)).to(tt[dt])
        return t.cuda(), t.to(torch.float64).numpy()
    if dt == "bf16":
        t = torch.from_numpy(np.ascontiguousarray(vals, np.float32)).to(torch.bfloat16)
        return t.cuda(), t.to(torch.float64).numpy()
    f8 = torch.from_numpy(np.ascontiguousarray(vals, np.float32)).to(torch.float8_e4m3fn)
    return f8.view(torch.uint8).cuda(), f8.to(torch.float64).numpy()


@pytest.mark.parametrize("case", ["A", "B"])
@pytest.mark.parametrize("real_dt,rep_dt", [("f32", "u8"), ("f64", "i8"), ("bf16", "i32"),
                                            ("f32", "e4m3"), ("f32", "f32")])
@pytest.mark.parametrize("n", [384, 201])
def test_fp8_storage_dtypes(case, real_dt, rep_dt, n):
    """Every element size into both conversions: n = 384 takes the vector
    load paths, n = 201 the per-element ones.  Rep-factors 0..16 and some
    larger integral E4M3 values (18, 24, 448)."""
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for
    rng = np.random.default_rng(n + len(real_dt + rep_dt) + (case == "B"))
    real = rng.uniform(-1, 1, size=(n, n)) * (rng.random((n, n)) < 0.8)
    rep = rng.integers(0, 17, size=(n, n)).astype(np.int64)
    if rep_dt not in ("i8", "u8"):
        rep[rng.random((n, n)) < 0.01] = 18
        rep[0, :3] = (24, 448, 448)
    if case == "A":
        (Xt, Xv), (Yt, Yv) = _stored(real, real_dt), _stored(rep, rep_dt)
        Yv = Yv.astype(np.int64)
        xd, yd = real_dt, rep_dt
    else:
        (Xt, Xv), (Yt, Yv) = _stored(rep, rep_dt), _stored(real, real_dt)
        Xv = Xv.astype(np.int64)
        xd, yd = rep_dt, real_dt
    inst = W.Instance(case, Xv, Yv, x_dtype=xd, y_dtype=yd, z_dtype="f32", target="fp32")
    Z = torch.full((n, n), float("nan"), device="cuda")
    p = Plan(desc_for(inst, variant=FP8))
    p(Xt, Yt, Z)
    p.sync()
    check(inst, Z.cpu().numpy())


@pytest.mark.parametrize("case", ["A", "B"])
def test_fp8_power_of_two_scaling_is_exact(case):
    """Each row of the split operand carries its own power-of-two scale, so
    multiplying a row of X (Case A) or a column of Y (Case B) by 2^e
    multiplies the matching row or column of Z by exactly 2^e: the same
    bits up to the exponent, for e from -90 to 90.  All-zero rows and
    columns give zeros."""
    rng = np.random.default_rng(5 if case == "A" else 6)
    n = 300
    real = rng.uniform(-1, 1, size=(n, n)).astype(np.float32)
    rep = rng.integers(0, 17, size=(n, n)).astype(np.int32)
    e = rng.integers(-90, 91, size=n)
    e[:4] = (-90, 90, 0, 1)
    scale = np.ldexp(1.0, e)
    zero = [7, 100]
    if case == "A":
        real[zero, :] = 0
        scaled = (real * scale[:, None]).astype(np.float32)
        base = W.Instance("A", real, rep, x_dtype="f32", y_dtype="i32")
        big = W.Instance("A", scaled, rep, x_dtype="f32", y_dtype="i32")
    else:
        real[:, zero] = 0
        scaled = (real * scale[None, :]).astype(np.float32)
        base = W.Instance("B", rep, real, x_dtype="i32", y_dtype="f32")
        big = W.Instance("B", rep, scaled, x_dtype="i32", y_dtype="f32")
    Z0, _ = run_gpu(base, variant=FP8)
    Z1, _ = run_gpu(big, variant=FP8)
    expect = Z0 * (scale[:, None] if case == "A" else scale[None, :])
    assert np.array_equal(Z1, expect.astype(np.float32))
    if case == "A":
        assert np.all(Z1[zero, :] == 0)
    else:
        assert np.all(Z1[:, zero] == 0)
    check(base, Z0)
    # The element bound scales with each row (column): every element of the
    # scaled product meets it too.
    check(big, Z1)


@pytest.mark.parametrize("case", ["A", "B"])
def test_fp8_rep_not_held_in_e4m3_is_reported(case):
    """17 has no E4M3 encoding (5 significant bits): the call records
    AFMM_ERR_OVERFLOW_RISK and afmm_plan_sync raises it."""
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    rng = np.random.default_rng(3)
    n = 160
    real = torch_of(rng.uniform(-1, 1, size=(n, n)).astype(np.float32))
    rep = rng.integers(0, 17, size=(n, n)).astype(np.int32)
    rep[5, 9] = 17
    rep = torch_of(rep)
    Z = torch.empty((n, n), dtype=torch.float32, device="cuda")
    if case == "A":
        p = Plan(make_desc(n, "A", "f32", "i32", "f32", "fp32", variant=FP8))
        p(real, rep, Z)
    else:
        p = Plan(make_desc(n, "B", "i32", "f32", "f32", "fp32", variant=FP8))
        p(rep, real, Z)
    with pytest.raises(AfmmError) as e:
        p.sync()
    assert e.value.status == 4          # AFMM_ERR_OVERFLOW_RISK


@pytest.mark.parametrize("case", ["A", "B"])
def test_fp8_non_finite_real_value_is_reported(case):
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    rng = np.random.default_rng(4)
    n = 130
    real = rng.uniform(-1, 1, size=(n, n)).astype(np.float32)
    real[17, 3] = np.inf
    rep = torch_of(rng.integers(0, 9, size=(n, n)).astype(np.int32))
    Z = torch.empty((n, n), dtype=torch.float32, device="cuda")
    if case == "A":
        p = Plan(make_desc(n, "A", "f32", "i32", "f32", "fp32", variant=FP8))
        p(torch_of(real), rep, Z)
    else:
        p = Plan(make_desc(n, "B", "i32", "f32", "f32", "fp32", variant=FP8))
        p(rep, torch_of(real), Z)
    with pytest.raises(AfmmError) as e:
        p.sync()
    assert e.value.status == 4


def test_fp8_leading_dimensions():
    """Padded rows on all three matrices; ldz = n + 5 takes the aligned
    product buffer and the 2-D copy; padding columns of Z untouched."""
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(8)
    n, pad = 131, 9
    Xb = rng.uniform(-1, 1, size=(n, n + pad)).astype(np.float32)
    Yb = rng.integers(0, 9, size=(n, n + pad + 3)).astype(np.int32)
    Zb = torch.full((n, n + 5), 7.0, dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "A", "f32", "i32", "f32", "fp32", variant=FP8,
                       ldx=n + pad, ldy=n + pad + 3, ldz=n + 5))
    p(torch_of(Xb), torch_of(Yb), Zb)
    p.sync()
    Z = Zb.cpu().numpy()
    check(W.Instance("A", Xb[:, :n], Yb[:, :n], x_dtype="f32", y_dtype="i32"), Z[:, :n])
    assert np.all(Z[:, n:] == 7.0)


@pytest.mark.parametrize("case", ["A", "B"])
def test_fp8_host_buffers_pipelined(case):
    """Host X, Y, Z: the transfers are pipelined with the products by row
    blocks; the result is bit-identical to the device-resident call."""
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for
    wl = "caseA_n8192_e4m3" if case == "A" else "caseB_n4096_f32"
    inst = W.make(wl, n=1500, seed=23)
    Zd, _ = run_gpu(inst, variant=FP8)
    check(inst, Zd, sample_rows(inst.n, 16))
    Xs = inst.x_store if inst.x_store is not None else inst.X
    Ys = inst.y_store if inst.y_store is not None else inst.Y
    p = Plan(desc_for(inst, variant=FP8))
    Xh = torch.from_numpy(np.ascontiguousarray(Xs)).pin_memory()
    Yh = torch.from_numpy(np.ascontiguousarray(Ys)).pin_memory()
    Zh = torch.full((inst.n, inst.n), float("nan")).pin_memory()
    p(Xh, Yh, Zh)
    p.sync()
    assert np.array_equal(Zh.numpy(), Zd)


def test_fp8_repeated_calls_replay_a_graph():
    from paper_1308_2400_gb300 import Plan
    from _helpers import desc_for, gpu_operands
    inst = W.make("caseA_n8192_e4m3", n=300, seed=9)
    p = Plan(desc_for(inst, variant=FP8))
    X, Y = gpu_operands(inst)
    Z = torch.empty((300, 300), dtype=torch.float32, device="cuda")
    outs = []
    for _ in range(4):
        p(X, Y, Z)
        p.sync()
        outs.append(Z.clone())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    check(inst, outs[0].cpu().numpy())


def test_fp8_error_between_two_and_three_bf16_slices():
    """About 20 significant bits per value: well inside the FP32 bar and
    far below the two-slice BF16 form (16 bits)."""
    inst = W.make("caseA_n8192_e4m3", n=1024, seed=3)
    Z8, _ = run_gpu(inst, variant=FP8)
    Z2, _ = run_gpu(inst, variant=2)
    R = oracle_rows(inst)
    e8, e2 = rel_fro(Z8, R), rel_fro(Z2, R)
    assert e8 < 1e-6 and e8 < e2 / 2


def test_fp8_empty_problem():
    """n = 0: nothing to do, no error, for either case."""
    from paper_1308_2400_gb300 import Plan, make_desc
    for case, xd, yd in (("A", "f32", "e4m3"), ("B", "i32", "f32")):
        p = Plan(make_desc(0, case, xd, yd, "f32", "fp32", variant=FP8))
        e = torch.empty((0, 0), dtype=torch.float32, device="cuda")
        p(e, e, e)
        p.sync()
        assert p.info["variant"] == FP8
        p.close()
