"""The C ABI without a GPU: the library loads, exports every entry point
include/afmm.h declares, and validates descriptors on the host."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "afmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(afmm_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1308_2400_gb300 import _build
    return ctypes.CDLL(_build.build())


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name


def test_binding_exposes_same_names():
    import paper_1308_2400_gb300 as P
    for name in declared_functions():
        assert hasattr(P.afmm, name), name


def test_binding_constants_match_header():
    """Every AFMM_VARIANT_, AFMM_FLAG_ and AFMM_ERR_ value the header
    defines has the same value in the Python binding."""
    import paper_1308_2400_gb300 as P
    src = open(os.path.join(ROOT, "include", "afmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    found = re.findall(r"\b(AFMM_(?:VARIANT|FLAG|ERR)_[A-Z0-9_]+)\s*=\s*(-?(?:0x)?[0-9A-Fa-f]+)u?",
                       src)
    assert len(found) >= 20
    for name, val in found:
        if name.endswith("COUNT_"):
            continue
        assert getattr(P.afmm, name) == int(val, 0), name


def test_status_strings():
    import paper_1308_2400_gb300 as P
    assert P.afmm_status_string(0) == "AFMM_OK"
    assert P.afmm_status_string(3) == "AFMM_ERR_NEGATIVE_REP"
    assert P.afmm_status_string(12345) == "AFMM_ERR_UNKNOWN"
    assert P.afmm_version() >= 100


@pytest.mark.parametrize("kw", [
    dict(n=-1),
    dict(case="A", x_dtype="f32", y_dtype="f64"),          # real Rep-factors
    dict(target="exact", x_dtype="f32", y_dtype="i8", z_dtype="i32"),
    dict(target="fp64", z_dtype="f32"),
    dict(target="fp32", z_dtype="f64"),
    dict(ldx=3),                                            # ldx < n
    dict(variant=99),
])
def test_invalid_descriptors_are_rejected(kw):
    import paper_1308_2400_gb300 as P
    base = dict(n=16, case="A", x_dtype="f32", y_dtype="i32", z_dtype="f32",
                target="fp32")
    base.update(kw)
    with pytest.raises(P.AfmmError) as e:
        P.afmm_plan_create(P.make_desc(**base))
    assert e.value.status == P.afmm.AFMM_ERR_INVALID_ARG


def test_planner_choices_and_workspace():
    import paper_1308_2400_gb300 as P
    A = P.afmm
    h = P.afmm_plan_create(P.make_desc(256, "A", "f64", "i32", "f64", "fp64"))
    info = P.afmm_get_info(h)
    assert info["variant"] == A.AFMM_VARIANT_SIMT_F64SLICE
    assert info["slices"] * info["slice_bits"] == 56
    assert P.afmm_plan_workspace_size(h) > 8 * 256 * 256
    P.afmm_plan_destroy(h)
    h = P.afmm_plan_create(P.make_desc(64, "A", "i8", "i8", "i32", "exact"))
    assert P.afmm_get_info(h)["variant"] == A.AFMM_VARIANT_SIMT_EXACT
    P.afmm_plan_destroy(h)
    # an exact target whose int32 sums could overflow is refused up front
    with pytest.raises(P.AfmmError) as e:
        P.afmm_plan_create(P.make_desc(1 << 17, "A", "i8", "i8", "i32",
                                       "exact"))
    assert e.value.status == A.AFMM_ERR_OVERFLOW_RISK
    # a variant that does not serve the target is refused
    with pytest.raises(P.AfmmError) as e:
        P.afmm_plan_create(P.make_desc(64, "A", "f32", "i32", "f32", "fp32",
                                       variant=A.AFMM_VARIANT_SIMT_EXACT))
    assert e.value.status == A.AFMM_ERR_UNSUPPORTED


def test_real_by_real_descriptors():
    """Two real factors (no Rep-factor): FP32 target only, and only the
    CUDA-core form or the two-sided tensor-core split serve them."""
    import paper_1308_2400_gb300 as P
    A = P.afmm
    for kw in (dict(target="fp64", z_dtype="f64"), dict(z_dtype="f64"),
               dict(x_dtype="e4m3")):
        base = dict(n=64, case="REAL", x_dtype="f32", y_dtype="f64", z_dtype="f32",
                    target="fp32")
        base.update(kw)
        with pytest.raises(P.AfmmError) as e:
            P.afmm_plan_create(P.make_desc(**base))
        assert e.value.status == A.AFMM_ERR_INVALID_ARG
    h = P.afmm_plan_create(P.make_desc(64, "REAL", "f32", "f64", "f32", "fp32",
                                       variant=A.AFMM_VARIANT_SIMT_F32))
    assert P.afmm_get_info(h)["variant"] == A.AFMM_VARIANT_SIMT_F32
    P.afmm_plan_destroy(h)
    for kase, v in (("REAL", A.AFMM_VARIANT_TC_FP8X4), ("REAL", A.AFMM_VARIANT_TC_BF16X3),
                    ("A", A.AFMM_VARIANT_TC_BF16X3X3), ("REAL", A.AFMM_VARIANT_TC_F16X2)):
        with pytest.raises(P.AfmmError) as e:
            P.afmm_plan_create(P.make_desc(64, kase, "f32", "i32", "f32", "fp32",
                                           variant=v))
        assert e.value.status == A.AFMM_ERR_UNSUPPORTED


def test_lent_workspace_is_checked():
    """A lent workspace smaller than the plan needs, or off a 256-byte
    boundary, is refused on the host before any device work (the pointer
    is never dereferenced here); a large enough aligned one is taken."""
    import paper_1308_2400_gb300 as P
    A = P.afmm
    h = P.afmm_plan_create(P.make_desc(256, "A", "f64", "i32", "f64", "fp64"))
    need = P.afmm_plan_workspace_size(h)
    assert need > 0
    base = 1 << 40                                   # an address, not memory
    with pytest.raises(P.AfmmError) as e:
        P.afmm_plan_set_workspace(h, base, need - 1)
    assert e.value.status == A.AFMM_ERR_INVALID_ARG
    with pytest.raises(P.AfmmError) as e:
        P.afmm_plan_set_workspace(h, base + 64, need)
    assert e.value.status == A.AFMM_ERR_INVALID_ARG
    P.afmm_plan_set_workspace(h, base, need)
    P.afmm_plan_destroy(h)                           # does not free a lent buffer


def test_null_arguments(lib):
    import paper_1308_2400_gb300 as P
    assert lib.afmm_plan_create(None, None) == P.afmm.AFMM_ERR_INVALID_ARG
    assert lib.afmm_plan_destroy(None) == 0
    assert lib.afmm_mul_caseA(None, None, None, None, None) == \
        P.afmm.AFMM_ERR_INVALID_ARG
