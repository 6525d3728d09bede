"""Python binding of libafmm (include/afmm.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name.  Pointers may
be torch tensors (device or host), numpy arrays (host) or plain integers;
streams may be ``torch.cuda.Stream`` objects, raw handles or ``None`` (the
current torch stream).  A status other than AFMM_OK raises ``AfmmError``.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1308_2400_gb300._build``); importing this module without
it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import _build

# ------------------------------------------------------------------ constants
AFMM_OK = 0
AFMM_ERR_INVALID_ARG = 1
AFMM_ERR_UNSUPPORTED = 2
AFMM_ERR_NEGATIVE_REP = 3
AFMM_ERR_OVERFLOW_RISK = 4
AFMM_ERR_OOM = 5
AFMM_ERR_CUDA = 6
AFMM_ERR_TIMEOUT = 7
AFMM_ERR_NO_DEVICE = 8
AFMM_ERR_NONINTEGER_REP = 9

AFMM_CASE_A, AFMM_CASE_B, AFMM_CASE_REAL = 0, 1, 2
AFMM_F64, AFMM_F32, AFMM_BF16, AFMM_E4M3, AFMM_I32, AFMM_I8, AFMM_U8 = range(7)
AFMM_TARGET_FP32, AFMM_TARGET_FP64, AFMM_TARGET_EXACT = 0, 1, 2
AFMM_VARIANT_AUTO = -1
AFMM_VARIANT_SIMT_F32 = 0
AFMM_VARIANT_TC_BF16X3 = 1
AFMM_VARIANT_TC_BF16X2 = 2
AFMM_VARIANT_SIMT_F64SLICE = 3
AFMM_VARIANT_SIMT_EXACT = 4
AFMM_VARIANT_TC_EXACT = 5
AFMM_VARIANT_SPARSE = 6
AFMM_VARIANT_TC_FP8X4 = 7
AFMM_VARIANT_TC_BF16X3X3 = 8
AFMM_VARIANT_TC_BF16X3_N128 = 9
AFMM_VARIANT_TC_F16X2 = 10
AFMM_VARIANT_TC_EXACT_F8 = 11
AFMM_FLAG_VALIDATE = 0x1
AFMM_FLAG_FUSED_SPLIT = 0x2

VARIANT_NAMES = {
    AFMM_VARIANT_SIMT_F32: "simt_f32", AFMM_VARIANT_TC_BF16X3: "tc_bf16x3",
    AFMM_VARIANT_TC_BF16X2: "tc_bf16x2",
    AFMM_VARIANT_SIMT_F64SLICE: "simt_f64slice",
    AFMM_VARIANT_SIMT_EXACT: "simt_exact", AFMM_VARIANT_TC_EXACT: "tc_exact",
    AFMM_VARIANT_SPARSE: "sparse", AFMM_VARIANT_TC_FP8X4: "tc_fp8x4",
    AFMM_VARIANT_TC_BF16X3X3: "tc_bf16x3x3",
    AFMM_VARIANT_TC_BF16X3_N128: "tc_bf16x3_n128",
    AFMM_VARIANT_TC_F16X2: "tc_f16x2",
    AFMM_VARIANT_TC_EXACT_F8: "tc_exact_f8",
}
CASE_CODES = {"A": AFMM_CASE_A, "B": AFMM_CASE_B, "REAL": AFMM_CASE_REAL}
DTYPE_CODES = {"f64": AFMM_F64, "f32": AFMM_F32, "bf16": AFMM_BF16,
               "e4m3": AFMM_E4M3, "i32": AFMM_I32, "i8": AFMM_I8,
               "u8": AFMM_U8}
TARGET_CODES = {"fp32": AFMM_TARGET_FP32, "fp64": AFMM_TARGET_FP64,
                "exact": AFMM_TARGET_EXACT}


class afmm_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ldx", ctypes.c_int64),
                ("ldy", ctypes.c_int64), ("ldz", ctypes.c_int64),
                ("kase", ctypes.c_int32), ("x_dtype", ctypes.c_int32),
                ("y_dtype", ctypes.c_int32), ("z_dtype", ctypes.c_int32),
                ("target", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved_", ctypes.c_int32),
                ("d1", ctypes.c_double), ("d2", ctypes.c_double),
                ("mu_prime", ctypes.c_double), ("rep_max", ctypes.c_double),
                ("base_max", ctypes.c_double)]


class afmm_info(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("slice_bits", ctypes.c_int32), ("k_split", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_uint64),
                ("d1", ctypes.c_double), ("d2", ctypes.c_double),
                ("mu_prime", ctypes.c_double), ("mu", ctypes.c_double),
                ("rep_max", ctypes.c_double),
                ("expected_additions", ctypes.c_double)]


class afmm_counters(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("timed_launches", ctypes.c_int64), ("timed_ms", ctypes.c_double),
                ("main_kernel_ctas", ctypes.c_int32), ("reserved_", ctypes.c_int32),
                ("simt_k_tiles", ctypes.c_int64)]


AFMM_DISPATCH_FEATURES = 10


class afmm_mlp_shape(ctypes.Structure):
    _fields_ = [("features", ctypes.c_int32), ("hidden", ctypes.c_int32),
                ("outputs", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class AfmmError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        msg = status_name(status)
        detail = ""
        try:
            detail = _lib().afmm_last_error_detail().decode()
        except Exception:  # pragma: no cover - best effort
            pass
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))


_LIB = None
_VP = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(
                f"libafmm.so is not built ({_build.LIB}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(_build.LIB)
        st = ctypes.c_int
        sig = {
            "afmm_status_string": ([st], ctypes.c_char_p),
            "afmm_last_error_detail": ([], ctypes.c_char_p),
            "afmm_version": ([], ctypes.c_int),
            "afmm_plan_create": ([ctypes.POINTER(_VP), ctypes.POINTER(afmm_desc)], st),
            "afmm_plan_destroy": ([_VP], st),
            "afmm_plan_workspace_size": ([_VP, ctypes.POINTER(ctypes.c_size_t)], st),
            "afmm_plan_set_workspace": ([_VP, _VP, ctypes.c_size_t], st),
            "afmm_mul_caseA": ([_VP, _VP, _VP, _VP, _VP], st),
            "afmm_mul_caseB": ([_VP, _VP, _VP, _VP, _VP], st),
            "afmm_mul_real": ([_VP, _VP, _VP, _VP, _VP], st),
            "afmm_mul_rows": ([_VP, ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP, _VP], st),
            "afmm_plan_sync": ([_VP, _VP], st),
            "afmm_get_info": ([_VP, ctypes.POINTER(afmm_info)], st),
            "afmm_plan_enable_kernel_timing": ([_VP, ctypes.c_int], st),
            "afmm_plan_counters": ([_VP, ctypes.POINTER(afmm_counters)], st),
            "afmm_selftest_bounded_wait": ([ctypes.c_uint64, _VP], st),
            "afmm_dispatch_features": ([ctypes.POINTER(afmm_desc),
                                        ctypes.POINTER(ctypes.c_float)], st),
            "afmm_mlp_param_count": ([ctypes.POINTER(afmm_mlp_shape)], ctypes.c_int64),
            "afmm_mlp_work_floats": ([ctypes.POINTER(afmm_mlp_shape), ctypes.c_int],
                                     ctypes.c_int64),
            "afmm_mlp_forward": ([ctypes.POINTER(afmm_mlp_shape), _VP, _VP, ctypes.c_int,
                                  _VP, _VP, _VP], st),
            "afmm_mlp_loss_grad": ([ctypes.POINTER(afmm_mlp_shape), _VP, _VP, _VP, _VP,
                                    ctypes.c_int, ctypes.c_float, _VP, _VP, _VP, _VP], st),
            "afmm_mlp_adam": ([ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_int, _VP], st),
            "afmm_set_dispatch_model": ([ctypes.POINTER(afmm_mlp_shape), _VP, _VP, _VP,
                                         _VP], st),
            "afmm_dispatch_variant": ([ctypes.POINTER(afmm_desc)], ctypes.c_int32),
            "afmm_batched_sync": ([ctypes.c_int, ctypes.POINTER(afmm_desc), _VP], st),
            "afmm_mul_noalloc": ([ctypes.POINTER(afmm_desc), _VP, _VP, _VP, _VP], st),
            "afmm_mul_batched": ([ctypes.c_int, ctypes.POINTER(afmm_desc),
                                  ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                  ctypes.POINTER(_VP), _VP], st),
            "afmm_error_norm_workspace_size": ([ctypes.c_int64, ctypes.c_int64],
                                               ctypes.c_size_t),
            "afmm_error_norm": ([_VP, ctypes.c_int32, ctypes.c_int64, _VP,
                                 ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_int64, _VP,
                                 ctypes.POINTER(ctypes.c_double), _VP], st),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _LIB = lib
    return _LIB


def status_name(s: int) -> str:
    try:
        return _lib().afmm_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


def _check(rc: int, where: str) -> None:
    if rc != AFMM_OK:
        raise AfmmError(rc, where)


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() else None
    if hasattr(x, "ctypes"):  # numpy
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> Optional[int]:
    if s is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream or None
        return None
    if isinstance(s, int):
        return s or None
    return s.cuda_stream or None


# ------------------------------------------------------------------ C ABI
def afmm_status_string(s: int) -> str:
    return status_name(s)


def afmm_last_error_detail() -> str:
    return _lib().afmm_last_error_detail().decode()


def afmm_version() -> int:
    return int(_lib().afmm_version())


def make_desc(n: int, case: str = "A", x_dtype="f32", y_dtype="f32",
              z_dtype="f32", target="fp32", variant: int = AFMM_VARIANT_AUTO,
              flags: int = 0, d1: float = -1.0, d2: float = -1.0,
              mu_prime: float = -1.0, ldx: int = 0, ldy: int = 0,
              ldz: int = 0, rep_max: float = -1.0,
              base_max: float = -1.0) -> afmm_desc:
    """Fill an ``afmm_desc`` from readable names ("A"/"B"/"REAL", "f32",
    "fp32")."""
    def code(v, table):
        return table[v] if isinstance(v, str) else int(v)
    return afmm_desc(n=int(n), ldx=int(ldx), ldy=int(ldy), ldz=int(ldz),
                     kase=code(str(case).upper() if isinstance(case, str) else case,
                               CASE_CODES),
                     x_dtype=code(x_dtype, DTYPE_CODES),
                     y_dtype=code(y_dtype, DTYPE_CODES),
                     z_dtype=code(z_dtype, DTYPE_CODES),
                     target=code(target, TARGET_CODES), variant=int(variant),
                     flags=int(flags), reserved_=0, d1=float(d1),
                     d2=float(d2), mu_prime=float(mu_prime),
                     rep_max=float(rep_max), base_max=float(base_max))


def afmm_plan_create(desc: afmm_desc) -> int:
    h = _VP()
    _check(_lib().afmm_plan_create(ctypes.byref(h), ctypes.byref(desc)),
           "afmm_plan_create")
    return h.value


def afmm_plan_destroy(plan: int) -> None:
    _check(_lib().afmm_plan_destroy(plan), "afmm_plan_destroy")


def afmm_plan_workspace_size(plan: int) -> int:
    b = ctypes.c_size_t()
    _check(_lib().afmm_plan_workspace_size(plan, ctypes.byref(b)),
           "afmm_plan_workspace_size")
    return int(b.value)


def afmm_plan_set_workspace(plan: int, ws, nbytes: int) -> None:
    _check(_lib().afmm_plan_set_workspace(plan, _ptr(ws), int(nbytes)),
           "afmm_plan_set_workspace")


def afmm_mul_caseA(plan: int, X, Y, Z, stream=None) -> None:
    _check(_lib().afmm_mul_caseA(plan, _ptr(X), _ptr(Y), _ptr(Z),
                                 _stream(stream)), "afmm_mul_caseA")


def afmm_mul_caseB(plan: int, X, Y, Z, stream=None) -> None:
    _check(_lib().afmm_mul_caseB(plan, _ptr(X), _ptr(Y), _ptr(Z),
                                 _stream(stream)), "afmm_mul_caseB")


def afmm_mul_real(plan: int, X, Y, Z, stream=None) -> None:
    _check(_lib().afmm_mul_real(plan, _ptr(X), _ptr(Y), _ptr(Z),
                                _stream(stream)), "afmm_mul_real")


def afmm_plan_sync(plan: int, stream=None) -> None:
    _check(_lib().afmm_plan_sync(plan, _stream(stream)), "afmm_plan_sync")


def afmm_get_info(plan: int) -> dict:
    info = afmm_info()
    _check(_lib().afmm_get_info(plan, ctypes.byref(info)), "afmm_get_info")
    return {f: getattr(info, f) for f, _ in afmm_info._fields_}


def afmm_plan_enable_kernel_timing(plan: int, enable: bool = True) -> None:
    _check(_lib().afmm_plan_enable_kernel_timing(plan, 1 if enable else 0),
           "afmm_plan_enable_kernel_timing")


def afmm_plan_counters(plan: int) -> dict:
    c = afmm_counters()
    _check(_lib().afmm_plan_counters(plan, ctypes.byref(c)),
           "afmm_plan_counters")
    return {f: getattr(c, f) for f, _ in afmm_counters._fields_
            if f != "reserved_"}


def afmm_selftest_bounded_wait(limit_ns: int, stream=None) -> int:
    """Status recorded by a kernel whose bounded wait must run out."""
    return int(_lib().afmm_selftest_bounded_wait(int(limit_ns), _stream(stream)))


def afmm_mul_noalloc(desc: afmm_desc, X, Y, Z, stream=None) -> None:
    """FP64-target product without any device allocation (n <= 256);
    device tensors only.  See include/afmm.h."""
    _check(_lib().afmm_mul_noalloc(ctypes.byref(desc), _ptr(X), _ptr(Y),
                                   _ptr(Z), _stream(stream)),
           "afmm_mul_noalloc")


def afmm_mul_rows(plan, r0: int, r1: int, Xrows, Y, Zrows, stream=None) -> None:
    """Rows [r0, r1) of Z from rows [r0, r1) of X and all of Y."""
    h = plan.handle if hasattr(plan, "handle") else plan
    _check(_lib().afmm_mul_rows(h, int(r0), int(r1), _ptr(Xrows), _ptr(Y), _ptr(Zrows),
                                _stream(stream)), "afmm_mul_rows")


def afmm_mul_batched(descs: Sequence[afmm_desc], X: Sequence, Y: Sequence,
                     Z: Sequence, stream=None) -> None:
    cnt = len(descs)
    arr = (afmm_desc * cnt)(*descs)
    px = (_VP * cnt)(*[_ptr(t) for t in X])
    py = (_VP * cnt)(*[_ptr(t) for t in Y])
    pz = (_VP * cnt)(*[_ptr(t) for t in Z])
    _check(_lib().afmm_mul_batched(cnt, arr, px, py, pz, _stream(stream)),
           "afmm_mul_batched")


def afmm_batched_sync(descs: Sequence[afmm_desc], stream=None) -> None:
    cnt = len(descs)
    arr = (afmm_desc * cnt)(*descs)
    _check(_lib().afmm_batched_sync(cnt, arr, _stream(stream)), "afmm_batched_sync")


def afmm_dispatch_features(desc: afmm_desc):
    out = (ctypes.c_float * AFMM_DISPATCH_FEATURES)()
    _check(_lib().afmm_dispatch_features(ctypes.byref(desc), out),
           "afmm_dispatch_features")
    return [float(v) for v in out]


def mlp_shape(features: int, hidden: int, outputs: int) -> afmm_mlp_shape:
    return afmm_mlp_shape(features=features, hidden=hidden, outputs=outputs,
                          reserved_=0)


def afmm_mlp_param_count(shape: afmm_mlp_shape) -> int:
    return int(_lib().afmm_mlp_param_count(ctypes.byref(shape)))


def afmm_mlp_work_floats(shape: afmm_mlp_shape, rows: int) -> int:
    return int(_lib().afmm_mlp_work_floats(ctypes.byref(shape), int(rows)))


def afmm_mlp_forward(shape, params, X, rows, P, work, stream=None) -> None:
    _check(_lib().afmm_mlp_forward(ctypes.byref(shape), _ptr(params), _ptr(X),
                                   int(rows), _ptr(P), _ptr(work), _stream(stream)),
           "afmm_mlp_forward")


def afmm_mlp_loss_grad(shape, params, X, T, M, rows, count, grads, work, loss,
                       stream=None) -> None:
    _check(_lib().afmm_mlp_loss_grad(ctypes.byref(shape), _ptr(params), _ptr(X),
                                     _ptr(T), _ptr(M), int(rows), float(count),
                                     _ptr(grads), _ptr(work), _ptr(loss),
                                     _stream(stream)), "afmm_mlp_loss_grad")


def afmm_mlp_adam(n, params, grads, m, v, lr, beta1, beta2, eps, step,
                  stream=None) -> None:
    _check(_lib().afmm_mlp_adam(int(n), _ptr(params), _ptr(grads), _ptr(m), _ptr(v),
                                float(lr), float(beta1), float(beta2), float(eps),
                                int(step), _stream(stream)), "afmm_mlp_adam")


def afmm_set_dispatch_model(shape, params, mean, scale, variants) -> None:
    """Host arrays (numpy float32 / int32); params None removes the model."""
    import numpy as np
    if params is None:
        _check(_lib().afmm_set_dispatch_model(None, None, None, None, None),
               "afmm_set_dispatch_model")
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = np.ascontiguousarray(mean, dtype=np.float32)
    s = np.ascontiguousarray(scale, dtype=np.float32)
    v = np.ascontiguousarray(variants, dtype=np.int32)
    _check(_lib().afmm_set_dispatch_model(ctypes.byref(shape), p.ctypes.data,
                                          m.ctypes.data, s.ctypes.data,
                                          v.ctypes.data), "afmm_set_dispatch_model")


def afmm_dispatch_variant(desc: afmm_desc) -> int:
    return int(_lib().afmm_dispatch_variant(ctypes.byref(desc)))


def afmm_error_norm_workspace_size(rows: int, cols: int) -> int:
    return int(_lib().afmm_error_norm_workspace_size(rows, cols))


def afmm_error_norm(Z, z_dtype, ldz, R, r_dtype, ldr, rows, cols,
                    workspace=None, stream=None):
    """(||Z - R||_F, ||R||_F, max|Z - R|) computed in FP64 on the GPU."""
    out = (ctypes.c_double * 3)()
    zc = DTYPE_CODES[z_dtype] if isinstance(z_dtype, str) else int(z_dtype)
    rc_ = DTYPE_CODES[r_dtype] if isinstance(r_dtype, str) else int(r_dtype)
    _check(_lib().afmm_error_norm(_ptr(Z), zc, int(ldz), _ptr(R), rc_,
                                  int(ldr), int(rows), int(cols),
                                  _ptr(workspace), out, _stream(stream)),
           "afmm_error_norm")
    return float(out[0]), float(out[1]), float(out[2])


# ------------------------------------------------------------------ helpers
class Plan:
    """Owning wrapper of an ``afmm_plan`` (destroyed with the object)."""

    def __init__(self, desc: afmm_desc):
        self.desc = desc
        self.handle = afmm_plan_create(desc)

    def close(self):
        if self.handle:
            afmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> dict:
        return afmm_get_info(self.handle)

    @property
    def variant_name(self) -> str:
        return VARIANT_NAMES.get(self.info["variant"], "?")

    def workspace_size(self) -> int:
        return afmm_plan_workspace_size(self.handle)

    def set_workspace(self, ws, nbytes: int) -> None:
        afmm_plan_set_workspace(self.handle, ws, nbytes)

    def __call__(self, X, Y, Z, stream=None) -> None:
        if self.desc.kase == AFMM_CASE_A:
            afmm_mul_caseA(self.handle, X, Y, Z, stream)
        elif self.desc.kase == AFMM_CASE_REAL:
            afmm_mul_real(self.handle, X, Y, Z, stream)
        else:
            afmm_mul_caseB(self.handle, X, Y, Z, stream)

    def sync(self, stream=None) -> None:
        afmm_plan_sync(self.handle, stream)

    def enable_kernel_timing(self, enable: bool = True) -> None:
        afmm_plan_enable_kernel_timing(self.handle, enable)

    def counters(self) -> dict:
        return afmm_plan_counters(self.handle)
