"""GB300 (sm_103a) implementation of the AFMM product of arXiv 1308.2400.

The compute path is ``libafmm.so`` (hand-written CUDA behind the C ABI in
``include/afmm.h``); this package only marshals arguments to it.
"""
from . import afmm  # noqa: F401
from .afmm import (AfmmError, Plan, afmm_batched_sync, afmm_error_norm,  # noqa: F401
                   afmm_error_norm_workspace_size, afmm_get_info,
                   afmm_mul_batched, afmm_mul_caseA, afmm_mul_real, afmm_mul_rows,
                   afmm_plan_counters, afmm_plan_enable_kernel_timing, afmm_mul_caseB,
                   afmm_plan_create, afmm_plan_destroy, afmm_plan_set_workspace,
                   afmm_plan_sync, afmm_plan_workspace_size,
                   afmm_status_string, afmm_version, make_desc)

__all__ = [n for n in dir() if n.startswith("afmm_")] + [
    "AfmmError", "Plan", "make_desc", "afmm"]
