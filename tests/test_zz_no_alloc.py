"""afmm_mul_noalloc: the FP64-target product that allocates nothing.

It is meant for callers that cannot call cudaMalloc (device memory held by
another allocator, loops that cannot afford an allocation's device
synchronisation, hosts that forbid allocating from their callbacks).  Its
scratch is a fixed array inside the library, shared by every call.  These
tests check its results element by element against the oracle (the Sec. 2
loops in FP64), two calls in a row against the plan entry point's
FP64-target form (the second call finding the first one's leftovers in the
array), that a call leaves the device's free memory unchanged, that bad
Rep-factors come back as an all-NaN Z, that padding columns of Z are not
touched, and that host pointers and oversized problems are refused.

This file is collected last so that, when it fails, a run stopping at the
first failure has already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest

import afmm_inputs as W
from _helpers import FP64_REL_FRO, rel_fro, torch_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _instance(case, n, seed):
    inst = W.make("caseA_n256_f64", n=n, seed=seed)
    if case == "B":
        inst = W.Instance("B", inst.Y.copy(), inst.X.T.copy(), x_dtype="i32",
                          y_dtype="f64", z_dtype="f64", target="fp64")
    return inst


def _desc(inst, variant=-1, ldz=0):
    from paper_1308_2400_gb300 import make_desc
    return make_desc(inst.n, inst.case, inst.x_dtype, inst.y_dtype, "f64",
                     "fp64", variant=variant, ldz=ldz)


def _with_plan(inst):
    """The existing entry point: a plan running the FP64-target form."""
    from paper_1308_2400_gb300 import Plan
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Z = torch.empty((inst.n, inst.n), dtype=torch.float64, device="cuda")
    p = Plan(_desc(inst, variant=3))
    p(X, Y, Z)
    p.sync()
    p.close()
    return Z.cpu().numpy()


def _no_alloc(inst, X=None, Y=None):
    from paper_1308_2400_gb300.afmm import afmm_mul_noalloc
    X = torch_of(inst.X) if X is None else X
    Y = torch_of(inst.Y) if Y is None else Y
    Z = torch.full((inst.n, inst.n), 123.0, dtype=torch.float64, device="cuda")
    afmm_mul_noalloc(_desc(inst), X, Y, Z)
    torch.cuda.synchronize()
    return Z.cpu().numpy()


def _oracle(inst):
    from oracle import afmm_case_a, afmm_case_b
    return (afmm_case_a if inst.case == "A" else afmm_case_b)(inst.X, inst.Y)[0]


def _element_bound(inst):
    """|Z - oracle| per element: the digit slices of the real factor miss
    each value by at most 2^-56 of its row's (Case A: X's row; Case B:
    Y's column) largest |value|; 1e-12 of that times the Rep-factor sums
    bounds the error with room for the FP64 recombination."""
    X = np.abs(inst.X.astype(np.float64))
    Y = np.abs(inst.Y.astype(np.float64))
    if inst.case == "A":
        return 1e-12 * X.max(axis=1, initial=0.0)[:, None] * Y.sum(axis=0)[None, :]
    return 1e-12 * X.sum(axis=1)[:, None] * Y.max(axis=0, initial=0.0)[None, :]


@pytest.mark.parametrize("case", ["A", "B"])
@pytest.mark.parametrize("n", [1, 7, 173, 256])
def test_matches_the_oracle_element_by_element(case, n):
    inst = _instance(case, n, seed=20 + n)
    Zn = _no_alloc(inst)
    R = _oracle(inst)
    assert np.all(np.isfinite(Zn))
    assert np.all(np.abs(Zn - R) <= _element_bound(inst) + 1e-300), (case, n)
    assert rel_fro(Zn, R) <= FP64_REL_FRO


@pytest.mark.parametrize("case", ["A", "B"])
def test_two_calls_in_a_row_match_the_plan_entry_point(case):
    first = _instance(case, 256, seed=11)      # the largest size it accepts
    second = _instance(case, 173, seed=12)     # ragged, after the first
    for inst in (first, second):
        Zn = _no_alloc(inst)
        Zp = _with_plan(inst)
        assert np.all(np.isfinite(Zn))
        assert rel_fro(Zn, Zp) <= FP64_REL_FRO, (case, inst.n)


def test_a_call_leaves_free_device_memory_unchanged():
    from paper_1308_2400_gb300.afmm import afmm_mul_noalloc
    inst = _instance("B", 200, seed=31)
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Z = torch.empty((200, 200), dtype=torch.float64, device="cuda")
    afmm_mul_noalloc(_desc(inst), X, Y, Z)        # warm-up: loads the code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        afmm_mul_noalloc(_desc(inst), X, Y, Z)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


@pytest.mark.parametrize("case", ["A", "B"])
@pytest.mark.parametrize("bad", [200, -3])
def test_bad_rep_factors_give_an_all_nan_z(case, bad):
    inst = _instance(case, 64, seed=41)
    rep = (inst.Y if case == "A" else inst.X).copy()
    rep[5, 9] = bad
    X = torch_of(inst.X if case == "A" else rep)
    Y = torch_of(rep if case == "A" else inst.Y)
    Zn = _no_alloc(inst, X, Y)
    assert np.all(np.isnan(Zn))
    assert np.all(np.isfinite(_no_alloc(inst)))   # the next good call is clean


def test_fractional_rep_factor_gives_an_all_nan_z():
    inst = _instance("A", 48, seed=42)
    Yf = inst.Y.astype(np.float32)
    Yf[3, 4] = 2.5
    inst_f = W.Instance("A", inst.X, Yf, x_dtype="f64", y_dtype="f32", z_dtype="f64",
                        target="fp64")
    Zn = _no_alloc(inst_f)
    assert np.all(np.isnan(Zn))


def test_padded_rows_of_z_keep_their_padding():
    from paper_1308_2400_gb300.afmm import afmm_mul_noalloc
    inst = _instance("A", 97, seed=51)
    ldz = 104
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Zb = torch.full((97, ldz), 777.0, dtype=torch.float64, device="cuda")
    afmm_mul_noalloc(_desc(inst, ldz=ldz), X, Y, Zb)
    torch.cuda.synchronize()
    Zh = Zb.cpu().numpy()
    assert np.all(Zh[:, 97:] == 777.0)
    R = _oracle(inst)
    assert np.all(np.abs(Zh[:, :97] - R) <= _element_bound(inst) + 1e-300)


def test_host_pointers_are_refused():
    from paper_1308_2400_gb300 import AfmmError
    from paper_1308_2400_gb300.afmm import AFMM_ERR_INVALID_ARG, afmm_mul_noalloc
    inst = _instance("A", 32, seed=61)
    Xh = np.ascontiguousarray(inst.X)
    Y = torch_of(inst.Y)
    Z = torch.empty((32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(AfmmError) as e:
        afmm_mul_noalloc(_desc(inst), Xh, Y, Z)
    assert e.value.status == AFMM_ERR_INVALID_ARG


def test_sizes_beyond_the_scratch_are_rejected():
    from paper_1308_2400_gb300 import AfmmError
    from paper_1308_2400_gb300.afmm import (AFMM_ERR_UNSUPPORTED,
                                            afmm_last_error_detail,
                                            afmm_mul_noalloc)
    inst = _instance("A", 257, seed=13)
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Z = torch.empty((257, 257), dtype=torch.float64, device="cuda")
    with pytest.raises(AfmmError) as e:
        afmm_mul_noalloc(_desc(inst), X, Y, Z)
    assert e.value.status == AFMM_ERR_UNSUPPORTED
    assert "256" in afmm_last_error_detail()
