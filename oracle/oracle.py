"""Python face of the C oracle for the AFMM product (arXiv 1308.2400, Sec. 2).

TEST INFRASTRUCTURE ONLY: the test suite, the package's smoke check and the
benchmark's CPU-baseline leg may import this module; the product path never
does.  It shares no code with the CUDA library.

The arithmetic lives in ``afmm_oracle.c`` (FP64 / int64 repeated addition in
the paper's i, k, j order, zero Base skipped).  This module only marshals
numpy arrays and states two closed forms of the paper:

* ``expected_additions``: E(A) = mu' * d1 * d2 * n^3 (Sec. 2.2);
* ``realised_parameters``: d1, d2 (fractions of non-zero entries of the pre
  and post factor, Sec. 1 and 2.2) and mu' / mu (mean of the non-zero
  Rep-factors / of all Rep-factors; mu = mu' * d, Sec. 2.2).
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Optional, Sequence, Tuple, Union

import numpy as np

from . import build as _build

__all__ = [
    "afmm_case_a", "afmm_case_b", "classical_ijk", "classical_ikj",
    "expected_additions", "realised_parameters", "oracle_threads",
    "set_oracle_threads", "rel_frobenius_error", "use_library",
]

_LIB = None
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def _load(path: str):
    lib = ctypes.CDLL(path)
    for name in ("afmm_oracle_caseA_f64", "afmm_oracle_caseB_f64",
                 "afmm_oracle_caseA_i64", "afmm_oracle_caseB_i64"):
        f = getattr(lib, name)
        f.argtypes = [_i64, _i64, _i64, _p, _p, _p, _p]
        f.restype = ctypes.c_int
    for name in ("afmm_oracle_caseA_f64_cols", "afmm_oracle_caseB_f64_cols",
                 "afmm_oracle_caseA_i64_cols", "afmm_oracle_caseB_i64_cols"):
        f = getattr(lib, name)
        f.argtypes = [_i64, _i64, _i64, _i64, _i64, _p, _p, _p, _p]
        f.restype = ctypes.c_int
    for name in ("afmm_classical_ijk_f64", "afmm_classical_ikj_f64"):
        f = getattr(lib, name)
        f.argtypes = [_i64, _i64, _i64, _p, _p, _p]
        f.restype = None
    lib.afmm_oracle_threads.restype = ctypes.c_int
    lib.afmm_oracle_set_threads.argtypes = [ctypes.c_int]
    return lib


class use_library:
    """Temporarily run the oracle from another build of ``afmm_oracle.c``.

    The test suite uses it to run the pins against copies of the oracle
    with a deliberately planted mistake.
    """

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _LIB
        self.saved = _LIB
        _LIB = _load(self.path)
        return _LIB

    def __exit__(self, *exc):
        global _LIB
        _LIB = self.saved
        return False


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = _load(_build.build())
    return _LIB


def oracle_threads() -> int:
    """Threads the oracle's row loop uses (OpenMP), 1 without OpenMP."""
    return int(_lib().afmm_oracle_threads())


def set_oracle_threads(t: int) -> None:
    _lib().afmm_oracle_set_threads(int(t))


RowSel = Union[None, Tuple[int, int], Sequence[int], np.ndarray]


def _row_runs(n: int, rows: RowSel) -> Tuple[np.ndarray, Iterable[Tuple[int, int]]]:
    """Resolve a row selection into the list of rows and contiguous runs."""
    if rows is None:
        idx = np.arange(n, dtype=np.int64)
    elif isinstance(rows, tuple) and len(rows) == 2:
        idx = np.arange(int(rows[0]), int(rows[1]), dtype=np.int64)
    else:
        idx = np.asarray(rows, dtype=np.int64).ravel()
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise ValueError("row index out of range")
    runs = []
    start = 0
    for t in range(1, idx.size + 1):
        if t == idx.size or idx[t] != idx[t - 1] + 1:
            runs.append((start, t))
            start = t
    return idx, runs


def _square(a: np.ndarray, name: str) -> int:
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError(f"{name} must be a square n x n matrix (Sec. 2)")
    return a.shape[0]


def _rep_factors(a: np.ndarray, name: str) -> np.ndarray:
    """Rep-factors are non-negative integers (Sec. 2 type lines, Sec. 2.1)."""
    a = np.asarray(a)
    if a.dtype.kind == "f":
        if not np.all(np.isfinite(a)) or not np.all(a == np.round(a)):
            raise ValueError(f"{name}: Rep-factors must be integers")
    elif a.dtype.kind not in "iu":
        raise ValueError(f"{name}: Rep-factors must be integers")
    a = np.ascontiguousarray(a, dtype=np.int64)
    if a.size and a.min() < 0:
        raise ValueError(f"{name}: Rep-factors must be non-negative")
    return a


def _run(fn, n, X, Y, rows, out_dtype, cols=None):
    """Rows `rows` of Z, restricted to the column window cols = (j0, j1)
    when given (each element formed exactly as in the full row)."""
    idx, runs = _row_runs(n, rows)
    j0, j1 = (0, n) if cols is None else (int(cols[0]), int(cols[1]))
    if not 0 <= j0 <= j1 <= n:
        raise ValueError("column window out of range")
    Z = np.zeros((idx.size, j1 - j0), dtype=out_dtype)
    total = 0
    adds = ctypes.c_uint64(0)
    for a, b in runs:
        i0, i1 = int(idx[a]), int(idx[b - 1]) + 1
        rc = fn(n, i0, i1, j0, j1, X.ctypes.data, Y.ctypes.data,
                Z[a:b].ctypes.data, ctypes.byref(adds))
        if rc != 0:
            raise ValueError("negative Rep-factor")
        total += adds.value
    return Z, total


def afmm_case_a(X: np.ndarray, Y: np.ndarray, rows: RowSel = None, cols=None):
    """Case A (Sec. 2): X real Base values, Y integer Rep-factors.

    Returns ``(Z_rows, additions)``: the selected rows of Z = X * Y formed
    by repeated addition (FP64, or exact int64 when X is integer-typed) and
    the number of additions performed on those rows; ``cols = (j0, j1)``
    restricts them to those columns.
    """
    n = _square(np.asarray(X), "X")
    if _square(np.asarray(Y), "Y") != n:
        raise ValueError("X and Y must have the same size n (Sec. 2)")
    Yi = _rep_factors(Y, "Y")
    lib = _lib()
    if np.asarray(X).dtype.kind in "iu":
        Xi = np.ascontiguousarray(X, dtype=np.int64)
        return _run(lib.afmm_oracle_caseA_i64_cols, n, Xi, Yi, rows, np.int64, cols)
    Xf = np.ascontiguousarray(X, dtype=np.float64)
    return _run(lib.afmm_oracle_caseA_f64_cols, n, Xf, Yi, rows, np.float64, cols)


def afmm_case_b(X: np.ndarray, Y: np.ndarray, rows: RowSel = None, cols=None):
    """Case B (Sec. 2): X integer Rep-factors, Y real Base values.

    A zero Base skips that single j (the reading under which the listing
    yields X * Y, Sec. 2.1).  Returns ``(Z_rows, additions)`` as above.
    """
    n = _square(np.asarray(X), "X")
    if _square(np.asarray(Y), "Y") != n:
        raise ValueError("X and Y must have the same size n (Sec. 2)")
    Xi = _rep_factors(X, "X")
    lib = _lib()
    if np.asarray(Y).dtype.kind in "iu":
        Yi = np.ascontiguousarray(Y, dtype=np.int64)
        return _run(lib.afmm_oracle_caseB_i64_cols, n, Xi, Yi, rows, np.int64, cols)
    Yf = np.ascontiguousarray(Y, dtype=np.float64)
    return _run(lib.afmm_oracle_caseB_f64_cols, n, Xi, Yf, rows, np.float64, cols)


def _classical(fn, X, Y, rows):
    n = _square(np.asarray(X), "X")
    Xf = np.ascontiguousarray(X, dtype=np.float64)
    Yf = np.ascontiguousarray(Y, dtype=np.float64)
    idx, runs = _row_runs(n, rows)
    Z = np.zeros((idx.size, n), dtype=np.float64)
    for a, b in runs:
        i0, i1 = int(idx[a]), int(idx[b - 1]) + 1
        fn(n, i0, i1, Xf.ctypes.data, Yf.ctypes.data, Z[a:b].ctypes.data)
    return Z


def classical_ijk(X, Y, rows: RowSel = None) -> np.ndarray:
    """Classical ijk multiply-add loop in FP64 (Table 1's "ijk")."""
    return _classical(_lib().afmm_classical_ijk_f64, X, Y, rows)


def classical_ikj(X, Y, rows: RowSel = None) -> np.ndarray:
    """Classical ikj multiply-add loop in FP64 (Table 1's "ikj")."""
    return _classical(_lib().afmm_classical_ikj_f64, X, Y, rows)


def expected_additions(mu_prime: float, d1: float, d2: float, n: int) -> float:
    """E(A) = mu' * d1 * d2 * n^3 (Sec. 2.2)."""
    return float(mu_prime) * float(d1) * float(d2) * float(n) ** 3


def realised_parameters(X: np.ndarray, Y: np.ndarray, case: str) -> dict:
    """d1, d2, mu' and mu of one instance as the paper defines them.

    d1, d2: fractions of non-zero entries of X and Y.  mu': mean of the
    non-zero Rep-factors (Y in case A, X in case B); mu: mean of all of them,
    equal to mu' * d of that factor (Sec. 2.2).
    """
    X = np.asarray(X)
    Y = np.asarray(Y)
    n2 = X.size
    d1 = float(np.count_nonzero(X)) / n2 if n2 else 0.0
    d2 = float(np.count_nonzero(Y)) / n2 if n2 else 0.0
    R = Y if case.upper() == "A" else X
    nz = np.count_nonzero(R)
    s = float(R.astype(np.float64).sum())
    mu_prime = s / nz if nz else 0.0
    mu = s / n2 if n2 else 0.0
    return {"d1": d1, "d2": d2, "mu_prime": mu_prime, "mu": mu}


def rel_frobenius_error(Z: np.ndarray, Z_ref: np.ndarray) -> float:
    """||Z - Z_ref||_F / ||Z_ref||_F in FP64 (0 when both are zero)."""
    Z = np.asarray(Z, dtype=np.float64)
    R = np.asarray(Z_ref, dtype=np.float64)
    den = float(np.sqrt(np.sum(R * R)))
    num = float(np.sqrt(np.sum((Z - R) ** 2)))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return num / den
