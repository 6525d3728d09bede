"""Error bounds of the operand splits that the GPU tests' element bounds use
(CPU tests; the rounding comes from PyTorch's own FP8 and BF16 conversions,
not from this library).

* FP8 form: a row scaled by the power of two that puts its largest |value|
  in [128, 256), cut into E4M3 slices q1, q2, q3 (round to nearest of the
  value and its residuals) and q4 (of the third residual times 2^12), leaves
  a rest of at most 2^-16 |v| or 2^-21 times the row's largest |value|.
* Split BF16: three round-to-nearest slices of an FP32 value sum to it
  exactly, and the slice products a real x real product leaves out,
  (2,3), (3,2), (3,3), stay below 2^-22 |x| |y|.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def e4m3(v: np.ndarray) -> np.ndarray:
    """E4M3 (fn) round to nearest even, through PyTorch's conversion."""
    t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32))
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def bf16(v: np.ndarray) -> np.ndarray:
    t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def test_e4m3_conversion_is_round_to_nearest():
    """The reference conversion itself: exact on E4M3 values, nearest (ties
    to even) between them."""
    assert np.array_equal(e4m3(np.array([1.0, 1.125, 17.0, 18.0, 448.0, 2.0 ** -9])),
                          [1.0, 1.125, 16.0, 18.0, 448.0, 2.0 ** -9])
    # 1 + 1/16 lies halfway between 1 and 1.125: ties to even (1).
    assert e4m3(np.array([1.0625]))[0] == 1.0
    assert e4m3(np.array([1.0626]))[0] == 1.125


def split4(rows: np.ndarray):
    """Slices of each row as the FP8 form cuts them (float64 arithmetic on
    FP32 inputs: every residual below is exact)."""
    amax = np.abs(rows).max(axis=1, keepdims=True)
    e = np.floor(np.log2(np.where(amax > 0, amax, 1.0)))
    v = rows * 2.0 ** (7 - e)
    r = v.copy()
    qs = []
    for _ in range(3):
        q = e4m3(r)
        qs.append(q)
        r = r - q
    q4 = e4m3(r * 2.0 ** 12)
    rest = r - q4 * 2.0 ** -12
    return v, qs + [q4], rest


@pytest.mark.parametrize("law", ["uniform", "normal", "wide"])
def test_fp8_four_slices_bound(law):
    rng = np.random.default_rng(7)
    n = 4096
    if law == "uniform":
        X = rng.uniform(-1, 1, (64, n))
    elif law == "normal":
        X = rng.standard_normal((64, n))
    else:                                    # values over 40 binades in a row
        X = rng.uniform(-1, 1, (64, n)) * 2.0 ** rng.uniform(-40, 0, (64, n))
    X = X.astype(np.float32).astype(np.float64)
    v, qs, rest = split4(X)
    assert np.all(np.abs(v) < 256)
    for q in qs:
        assert np.all(np.abs(q) <= 448)
    vmax = np.abs(v).max(axis=1, keepdims=True)
    bound = np.maximum(2.0 ** -16 * np.abs(v), 2.0 ** -21 * vmax)
    assert np.all(np.abs(rest) <= bound)
    # The truncation alone keeps a product inside the FP32 bar: about 3e-7
    # on the uniform and normal laws; rows spanning 40 binades reach 5.5e-7,
    # their small values keeping only the absolute part of the bound.
    Y = np.minimum(rng.poisson(3.0, (n, 32)), 16).astype(np.float64)
    exact = v @ Y
    approx = (qs[0] + qs[1] + qs[2] + qs[3] * 2.0 ** -12) @ Y
    err = np.linalg.norm(approx - exact) / np.linalg.norm(exact)
    assert err < (1e-6 if law == "wide" else 5e-7)


def test_three_e4m3_slices_miss_the_fp32_bar():
    """Three E4M3 slices (no rescaled fourth) miss the 1e-6 bar; this is
    why the form keeps four."""
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, (64, 2048)).astype(np.float32).astype(np.float64)
    v, qs, _ = split4(X)
    Y = np.minimum(rng.poisson(3.0, (2048, 32)), 16).astype(np.float64)
    exact = v @ Y
    three = (qs[0] + qs[1] + qs[2]) @ Y
    assert np.linalg.norm(three - exact) / np.linalg.norm(exact) > 1e-6


def test_bf16_three_slices_and_dropped_pairs():
    rng = np.random.default_rng(9)
    x = (rng.standard_normal(200_000) * 2.0 ** rng.uniform(-30, 30, 200_000)).astype(np.float32)
    y = (rng.standard_normal(200_000) * 2.0 ** rng.uniform(-30, 30, 200_000)).astype(np.float32)

    def slices(a):
        a = a.astype(np.float64)
        s1 = bf16(a)
        s2 = bf16(a - s1)
        s3 = bf16(a - s1 - s2)
        return s1, s2, s3

    x1, x2, x3 = slices(x)
    y1, y2, y3 = slices(y)
    assert np.array_equal(x1 + x2 + x3, x.astype(np.float64))
    assert np.array_equal(y1 + y2 + y3, y.astype(np.float64))
    dropped = np.abs(x2 * y3) + np.abs(x3 * y2) + np.abs(x3 * y3)
    assert np.all(dropped <= 2.0 ** -22 * np.abs(x.astype(np.float64) * y))
