"""Out-of-bounds writes (GPU tests, in place of a memory checker).

Every form runs with a lent workspace between two 64 KiB guard bands and
with Z inside a larger buffer: a guard row above and below and guard
columns to the right (ldz = n + 16).  After the call every guard byte must
be untouched, and the interior must match the oracle.  Ragged sizes put
partial tiles at every edge; Case B covers the transposed epilogue.
"""
from __future__ import annotations

import numpy as np
import pytest

import afmm_inputs as W
from _helpers import FP32_REL_FRO, FP64_REL_FRO, oracle_rows, rel_fro, torch_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 1 << 16
PAT = 0xA5

# name: (variant, case, x dtype, y dtype, z dtype, target)
FORMS = {
    "simt_f32_A": (0, "A", "f32", "i32", "f32", "fp32"),
    "tc_bf16x3_A": (1, "A", "f32", "i32", "f32", "fp32"),
    "tc_bf16x3_B": (1, "B", "i32", "f32", "f32", "fp32"),
    "tc_fp8x4_A": (7, "A", "f32", "i32", "f32", "fp32"),
    "tc_fp8x4_B": (7, "B", "i32", "f32", "f32", "fp32"),
    "sparse_B": (6, "B", "i32", "f32", "f32", "fp32"),
    "simt_f64slice_A": (3, "A", "f64", "i32", "f64", "fp64"),
    "simt_f64slice_B": (3, "B", "i32", "f64", "f64", "fp64"),
    "simt_exact_A": (4, "A", "i8", "i8", "i32", "exact"),
    "tc_exact_A": (5, "A", "i8", "i8", "i32", "exact"),
    "tc_exact_B": (5, "B", "i8", "i8", "i32", "exact"),
    "tc_bf16x3x3_real": (8, "REAL", "f32", "f32", "f32", "fp32"),
}


def operands(case, xd, yd, n, rng):
    def real(dt):
        v = rng.uniform(-1, 1, (n, n)) * (rng.random((n, n)) < 0.8)
        return v.astype(np.float64 if dt == "f64" else np.float32)

    def rep(dt):
        v = rng.integers(0, 16, (n, n)) * (rng.random((n, n)) < 0.7)
        return v.astype({"i32": np.int32, "i8": np.int8}[dt])

    if case == "REAL":
        return real(xd), real(yd)
    if xd == "i8" and yd == "i8":                      # exact: signed Base
        X = rng.integers(-127, 128, (n, n)).astype(np.int8)
        Y = rng.integers(0, 16, (n, n)).astype(np.int8)
        return (X, Y) if case == "A" else (Y, X)
    return (real(xd), rep(yd)) if case == "A" else (rep(xd), real(yd))


@pytest.mark.parametrize("n", [129, 300])
@pytest.mark.parametrize("form", sorted(FORMS))
def test_no_write_outside_z_and_workspace(form, n):
    _guarded_run(form, n)


@pytest.mark.parametrize("n", [641, 1283])
@pytest.mark.parametrize("form", ["tc_bf16x3_A", "tc_bf16x3_B", "tc_bf16x2_A",
                                  "tc_exact_A", "tc_exact_B"])
def test_large_ragged_tiles_write_only_z(form, n):
    """From n = 512 the split forms run on CTA pairs (256 x 256 tiles, the
    last round's tiles in 256 x 128 halves) and the exact form on 256 x 256
    tiles; ragged sizes leave partial tiles at the right and bottom edges."""
    _guarded_run(form, n)


FORMS["tc_bf16x2_A"] = (2, "A", "f32", "i32", "f32", "fp32")


def _guarded_run(form, n):
    from paper_1308_2400_gb300 import Plan, make_desc
    variant, case, xd, yd, zd, target = FORMS[form]
    rng = np.random.default_rng(n + len(form))
    X, Y = operands(case, xd, yd, n, rng)
    if form.startswith("sparse"):
        d = 3.0 / np.sqrt(n)
        X = (X * (rng.random((n, n)) < d)).astype(X.dtype)
        Y = (Y * (rng.random((n, n)) < d)).astype(Y.dtype)
    ldz = n + 16
    p = Plan(make_desc(n, case, xd, yd, zd, target, variant=variant, ldz=ldz,
                       d1=float(np.count_nonzero(X)) / n / n,
                       d2=float(np.count_nonzero(Y)) / n / n))
    assert p.info["variant"] == variant
    wsb = p.workspace_size()
    ws = torch.full((wsb + 2 * GUARD,), PAT, dtype=torch.uint8, device="cuda")
    p.set_workspace(ws[GUARD:], wsb)
    zt = {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32}[zd]
    fill = -7 if zd == "i32" else 7.0
    Zb = torch.full((n + 2, ldz), fill, dtype=zt, device="cuda")
    p(torch_of(X), torch_of(Y), Zb[1:n + 1])
    p.sync()
    w = ws.cpu().numpy()
    assert np.all(w[:GUARD] == PAT) and np.all(w[GUARD + wsb:] == PAT), form
    Zh = Zb.cpu().numpy()
    assert np.all(Zh[0] == fill) and np.all(Zh[n + 1] == fill), form
    assert np.all(Zh[1:n + 1, n:] == fill), form
    Z = Zh[1:n + 1, :n]
    if case == "REAL":
        from oracle import classical_ikj
        R = classical_ikj(X, Y)
    else:
        inst = W.Instance(case, X, Y, x_dtype=xd, y_dtype=yd, z_dtype=zd, target=target)
        R = oracle_rows(inst)
    if target == "exact":
        assert np.array_equal(Z.astype(np.int64), R)
    else:
        tol = FP64_REL_FRO if target == "fp64" else FP32_REL_FRO
        if variant == 2:
            tol = 1e-5           # two BF16 slices: short of FP32 by design
        assert rel_fro(Z, R) <= tol
    p.close()
