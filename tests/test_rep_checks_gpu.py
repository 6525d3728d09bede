"""Every form checks its Rep-factors on every call, with no flag set.

The paper types the Rep-factor as a non-negative integer (Sec. 2, the
INTEGER declarations of both listings; a negative count of additions has no
meaning in Sec. 2.1's argument).  Each product therefore reports a negative
Rep-factor as AFMM_ERR_NEGATIVE_REP and a non-integer one (NaN included) as
AFMM_ERR_NONINTEGER_REP through the plan's status word, and the next call
with valid inputs runs clean.  Negative Base values stay valid.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 70

# (variant, case, x dtype, y dtype, z dtype, target)
FORMS = [
    (0, "A", "f32", "i32", "f32", "fp32"),
    (0, "A", "f32", "f32", "f32", "fp32"),
    (0, "B", "i32", "f32", "f32", "fp32"),
    (1, "A", "f32", "e4m3", "f32", "fp32"),
    (1, "A", "f32", "f32", "f32", "fp32"),
    (1, "B", "f32", "f32", "f32", "fp32"),
    (1, "B", "i32", "f32", "f32", "fp32"),
    (2, "A", "f32", "bf16", "f32", "fp32"),
    (7, "A", "f32", "e4m3", "f32", "fp32"),
    (7, "B", "f32", "f32", "f32", "fp32"),
    (3, "A", "f64", "i32", "f64", "fp64"),
    (3, "B", "i32", "f64", "f64", "fp64"),
    (3, "A", "f64", "f32", "f64", "fp64"),
    (4, "A", "i8", "i8", "i32", "exact"),
    (4, "B", "i8", "i8", "i32", "exact"),
    (5, "A", "i8", "i8", "i32", "exact"),
    (5, "B", "i8", "i32", "i32", "exact"),
    (6, "A", "f32", "i32", "f32", "fp32"),
    (6, "B", "f32", "f32", "f32", "fp32"),
]

TORCH = {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32,
         "i8": torch.int8, "bf16": torch.bfloat16}


def _tensor(values, dt):
    t = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64))
    if dt == "e4m3":
        return t.to(torch.float32).to(torch.float8_e4m3fn).view(torch.uint8).cuda()
    return t.to(TORCH[dt]).cuda()


def _operands(case, xdt, ydt, rep_value):
    rng = np.random.default_rng(5)
    rep = rng.integers(0, 4, size=(N, N)).astype(np.float64)
    base = rng.integers(-3, 4, size=(N, N)).astype(np.float64)   # negatives allowed
    if rep_value is not None:
        rep[N - 1, 3] = rep_value
    X, Y = (base, rep) if case == "A" else (rep, base)
    return _tensor(X, xdt), _tensor(Y, ydt)


def _run(form, rep_value):
    from paper_1308_2400_gb300 import Plan, make_desc
    v, case, xdt, ydt, zdt, target = form
    X, Y = _operands(case, xdt, ydt, rep_value)
    Z = torch.empty((N, N), dtype={"f32": torch.float32, "f64": torch.float64,
                                   "i32": torch.int32}[zdt], device="cuda")
    p = Plan(make_desc(N, case, xdt, ydt, zdt, target, variant=v))
    try:
        p(X, Y, Z)
        p.sync()
    finally:
        p.close()


@pytest.mark.parametrize("form", FORMS, ids=lambda f: f"v{f[0]}-{f[1]}-{f[2]}-{f[3]}")
def test_negative_rep_factor_is_reported(form):
    from paper_1308_2400_gb300 import AfmmError
    from paper_1308_2400_gb300.afmm import AFMM_ERR_NEGATIVE_REP
    with pytest.raises(AfmmError) as e:
        _run(form, -2.0)
    assert e.value.status == AFMM_ERR_NEGATIVE_REP
    _run(form, None)                     # valid inputs: no error


@pytest.mark.parametrize("form", [f for f in FORMS if (f[3] if f[1] == "A" else f[2])
                                  in ("f32", "f64", "bf16")],
                         ids=lambda f: f"v{f[0]}-{f[1]}-{f[2]}-{f[3]}")
@pytest.mark.parametrize("bad", [0.5, float("nan")])
def test_non_integer_rep_factor_is_reported(form, bad):
    from paper_1308_2400_gb300 import AfmmError
    from paper_1308_2400_gb300.afmm import AFMM_ERR_NONINTEGER_REP
    with pytest.raises(AfmmError) as e:
        _run(form, bad)
    assert e.value.status == AFMM_ERR_NONINTEGER_REP
    _run(form, None)


def test_batched_reports_bad_rep_factors_on_both_routes():
    """A tensor-core instance with a negative Rep-factor comes back as NaN
    and a CUDA-core instance with a fractional FP32 one is reported; the
    batch's status names the error once and is then clear."""
    from paper_1308_2400_gb300 import afmm as A
    from paper_1308_2400_gb300 import AfmmError
    descs, Xs, Ys, Zs = [], [], [], []
    for t, (case, v, rep_value) in enumerate((("A", A.AFMM_VARIANT_TC_BF16X3, -1.0),
                                              ("B", A.AFMM_VARIANT_SIMT_F32, 2.5),
                                              ("A", A.AFMM_VARIANT_TC_BF16X3, None))):
        X, Y = _operands(case, "f32", "f32", rep_value)
        Xs.append(X)
        Ys.append(Y)
        Zs.append(torch.zeros((N, N), dtype=torch.float32, device="cuda"))
        descs.append(A.make_desc(N, case, "f32", "f32", "f32", "fp32", variant=v))
    A.afmm_mul_batched(descs, Xs, Ys, Zs)
    with pytest.raises(AfmmError) as e:
        A.afmm_batched_sync(descs)
    assert e.value.status in (A.AFMM_ERR_NEGATIVE_REP, A.AFMM_ERR_NONINTEGER_REP)
    assert torch.isnan(Zs[0]).all()
    assert torch.isfinite(Zs[2]).all()
    A.afmm_batched_sync(descs)           # reported once, then clear
