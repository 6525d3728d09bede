"""Real x real products (AFMM_CASE_REAL, afmm_mul_real) against the oracle's
classical FP64 product (GPU tests).

With no Rep-factor the product is the plain Z = X Y; the oracle is its
classical triple loop in FP64 (pinned against numpy's product in the CPU
suite).  The tensor-core form splits both factors into three BF16 slices
(x = x1 + x2 + x3 exactly for FP32 x, |x2| <= 2^-8 |x1|, |x3| <= 2^-16 |x1|)
and leaves out the slice products (2,3), (3,2), (3,3): at most
(2 * 2^-24 + 2^-32) |x| |y| per term, so per element

    |Z - XY|_ij <= 2^-22 (|X| |Y|)_ij + accumulation

the accumulation term being that of the one-sided split form.
"""
from __future__ import annotations

import numpy as np
import pytest

from _helpers import FP32_REL_FRO, U32, rel_fro, sample_rows, torch_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC_REAL = 8
SIMT = 0
RAGGED = [1, 7, 33, 127, 128, 129, 255, 257, 300, 513]


def oracle(X, Y, rows=None):
    from oracle import classical_ikj
    return classical_ikj(X, Y, rows)


def bound(X, Y, rows=None, variant=TC_REAL):
    Xa = np.abs(np.asarray(X, np.float64))
    if rows is not None:
        Xa = Xa[rows]
    XY = Xa @ np.abs(np.asarray(Y, np.float64))
    n = X.shape[0]
    if variant == TC_REAL:
        return (2.0 ** -22 + 2 * (2 * 2 * -(-n // 16) + 8) * U32) * XY + 1e-30
    return (32 + -(-n // 32) + 2) * U32 * XY + 1e-30


def run(X, Y, variant=-1, xd="f32", yd="f32", Xt=None, Yt=None):
    from paper_1308_2400_gb300 import Plan, make_desc
    n = X.shape[0]
    Xt = torch_of(X) if Xt is None else Xt
    Yt = torch_of(Y) if Yt is None else Yt
    Z = torch.full((n, n), float("nan"), device="cuda")
    p = Plan(make_desc(n, "REAL", xd, yd, "f32", "fp32", variant=variant))
    p(Xt, Yt, Z)
    p.sync()
    info = p.info
    p.close()
    return Z.cpu().numpy(), info


def check(X, Y, Z, rows=None, variant=TC_REAL):
    R = oracle(X, Y, rows)
    Zs = Z if rows is None else Z[rows]
    assert np.all(np.isfinite(Zs))
    err = rel_fro(Zs, R)
    assert err <= FP32_REL_FRO, err
    bad = np.abs(Zs.astype(np.float64) - R) > bound(X, Y, rows, variant)
    assert not bad.any(), int(bad.sum())
    return err


@pytest.mark.parametrize("n", RAGGED)
@pytest.mark.parametrize("variant", [TC_REAL, SIMT])
def test_real_ragged(variant, n):
    """Signed, zero-containing reals on both sides, every tile edge."""
    rng = np.random.default_rng(n + 7 * variant)
    X = (rng.uniform(-1, 1, (n, n)) * (rng.random((n, n)) < 0.8)).astype(np.float32)
    Y = rng.standard_normal((n, n)).astype(np.float32)
    Z, info = run(X, Y, variant)
    assert info["variant"] == variant
    check(X, Y, Z, variant=variant)


def test_real_full_size_sampled():
    rng = np.random.default_rng(11)
    n = 4096
    X = rng.standard_normal((n, n)).astype(np.float32)
    Y = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    Z, info = run(X, Y)
    assert info["variant"] == TC_REAL and info["slices"] == 3
    check(X, Y, Z, sample_rows(n, 16))


@pytest.mark.parametrize("xd,yd", [("f64", "bf16"), ("bf16", "f64"), ("i32", "f32"),
                                   ("f32", "i8")])
def test_real_storage_dtypes(xd, yd):
    n = 320
    rng = np.random.default_rng(len(xd + yd))
    vals = {"f64": lambda: rng.uniform(-1, 1, (n, n)),
            "f32": lambda: rng.uniform(-1, 1, (n, n)).astype(np.float32),
            "bf16": lambda: rng.uniform(-1, 1, (n, n)).astype(np.float32),
            "i32": lambda: rng.integers(-1000, 1001, (n, n)).astype(np.int32),
            "i8": lambda: rng.integers(-127, 128, (n, n)).astype(np.int8)}

    def stored(dt):
        v = vals[dt]()
        if dt == "bf16":
            t = torch.from_numpy(v).to(torch.bfloat16)
            return t.cuda(), t.to(torch.float64).numpy()
        return torch_of(v), np.asarray(v, np.float64)
    (Xt, Xv), (Yt, Yv) = stored(xd), stored(yd)
    Z, _ = run(Xv, Yv, TC_REAL, xd, yd, Xt, Yt)
    # FP64 inputs are rounded to FP32 first (the FP32 target needs no more):
    # add that rounding, u32 |x| per operand, to the bound.
    R = oracle(Xv, Yv)
    err = rel_fro(Z, R)
    assert err <= FP32_REL_FRO, err
    XY = np.abs(Xv) @ np.abs(Yv)
    assert np.all(np.abs(Z - R) <= bound(Xv, Yv) + 2 * U32 * XY)


def test_real_planner_and_entry_points():
    """AUTO picks the tensor-core form from n = 128 and the CUDA-core form
    below; a real x real plan runs only through afmm_mul_real, and the
    Rep-factor checks of the validating scan do not apply to it."""
    from paper_1308_2400_gb300 import AfmmError, Plan, make_desc
    from paper_1308_2400_gb300.afmm import afmm_mul_caseA
    rng = np.random.default_rng(3)
    for n, v in ((96, SIMT), (160, TC_REAL)):
        X = rng.uniform(-1, 1, (n, n)).astype(np.float32)
        Y = -rng.uniform(0.5, 1.5, (n, n)).astype(np.float32)   # negative, non-integer
        Z, info = run(X, Y)
        assert info["variant"] == v
        check(X, Y, Z, variant=v)
    p = Plan(make_desc(160, "REAL", "f32", "f32", "f32", "fp32", flags=1))
    Xt, Yt = torch_of(X), torch_of(Y)
    Zt = torch.empty((160, 160), dtype=torch.float32, device="cuda")
    p(Xt, Yt, Zt)
    p.sync()                           # no NEGATIVE_REP / NONINTEGER_REP
    assert p.info["d1"] == 1.0 and p.info["d2"] == 1.0
    with pytest.raises(AfmmError) as e:
        afmm_mul_caseA(p.handle, Xt, Yt, Zt)
    assert e.value.status == 1         # AFMM_ERR_INVALID_ARG
    p.close()


def test_real_host_buffers():
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(5)
    n = 600
    X = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    Y = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    Zd, _ = run(X, Y)
    p = Plan(make_desc(n, "REAL", "f32", "f32", "f32", "fp32"))
    Zh = torch.full((n, n), float("nan")).pin_memory()
    p(torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory(), Zh)
    p.sync()
    assert np.array_equal(Zh.numpy(), Zd)


def test_real_leading_dimensions():
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(6)
    n = 131
    Xb = rng.uniform(-1, 1, (n, n + 9)).astype(np.float32)
    Yb = rng.standard_normal((n, n + 3)).astype(np.float32)
    Zb = torch.full((n, n + 5), 7.0, dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "REAL", "f32", "f32", "f32", "fp32", ldx=n + 9, ldy=n + 3,
                       ldz=n + 5))
    p(torch_of(Xb), torch_of(Yb), Zb)
    p.sync()
    Z = Zb.cpu().numpy()
    check(np.ascontiguousarray(Xb[:, :n]), np.ascontiguousarray(Yb[:, :n]), Z[:, :n])
    assert np.all(Z[:, n:] == 7.0)


def test_real_repeated_calls_replay_a_graph():
    """From the third call on the same device buffers the product is
    replayed from a CUDA graph; replays give the eager call's bits and read
    the buffers' current contents."""
    from paper_1308_2400_gb300 import Plan, make_desc
    rng = np.random.default_rng(8)
    n = 300
    X = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    Y = rng.standard_normal((n, n)).astype(np.float32)
    Xt, Yt = torch_of(X), torch_of(Y)
    Z = torch.empty((n, n), dtype=torch.float32, device="cuda")
    p = Plan(make_desc(n, "REAL", "f32", "f32", "f32", "fp32"))
    outs = []
    for _ in range(4):
        p(Xt, Yt, Z)
        p.sync()
        outs.append(Z.clone())
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    check(X, Y, outs[0].cpu().numpy())
    X2 = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    Xt.copy_(torch_of(X2))
    p(Xt, Yt, Z)
    p.sync()
    check(X2, Y, Z.cpu().numpy())
    p.close()


@pytest.mark.parametrize("variant", [TC_REAL, SIMT])
def test_real_empty_problem(variant):
    from paper_1308_2400_gb300 import Plan, make_desc
    p = Plan(make_desc(0, "REAL", "f32", "f32", "f32", "fp32", variant=variant))
    e = torch.empty((0, 0), dtype=torch.float32, device="cuda")
    p(e, e, e)
    p.sync()
    assert p.info["variant"] == variant
    p.close()
