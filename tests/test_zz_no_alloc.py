"""afmm_mul_noalloc: the FP64-target product that allocates nothing.

It is meant for callers that cannot call cudaMalloc (device memory held by
another allocator, loops that cannot afford an allocation's device
synchronisation, hosts that forbid allocating from their callbacks).  Its
scratch is a fixed array inside the library, shared by every call, so
these tests check that two calls in a row -- the second one finding the
first one's leftovers in the array -- each match what the plan API's
FP64-target form returns for the same inputs, within the FP64-target
tolerance the other tests use (relative Frobenius error 1e-12).

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


def _desc(inst, variant=-1):
    from paper_1308_2400_gb300 import make_desc
    return make_desc(inst.n, inst.case, inst.x_dtype, inst.y_dtype, "f64",
                     "fp64", variant=variant)


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


def _no_alloc(inst):
    from paper_1308_2400_gb300.afmm import afmm_mul_noalloc
    X, Y = torch_of(inst.X), torch_of(inst.Y)
    Z = torch.full((inst.n, inst.n), 123.0, dtype=torch.float64, device="cuda")
    afmm_mul_noalloc(_desc(inst), X, Y, Z)
    torch.cuda.synchronize()
    return Z.cpu().numpy()


@pytest.mark.parametrize("case", ["A", "B"])
def test_two_calls_in_a_row_match_the_plan_entry_point(case):
    first = _instance(case, 256, seed=11)      # the largest size it accepts
    second = _instance(case, 173, seed=12)     # ragged, after the first
    for inst in (first, second):
        Zn = _no_alloc(inst)
        Zp = _with_plan(inst)
        assert np.all(np.isfinite(Zn))
        assert rel_fro(Zn, Zp) <= FP64_REL_FRO, (case, inst.n)


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
