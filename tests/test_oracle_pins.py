"""Pins of the CPU oracle against facts the paper and mathematics fix.

The oracle (``oracle/afmm_oracle.c``) follows the AFMM listings of Sec. 2.
These tests tie it to things other than itself:

* hand-worked examples under ``tests/golden/`` (Sec. 2 listings, Sec. 2.2
  count definition);
* brute force with exact rational arithmetic on tiny inputs, and the
  recursive-summation error bound for FP64 results;
* the classical multiply-add product through numpy (a library routine the
  oracle does not use), bit-exact on integer and dyadic inputs;
* the exact closed form of the addition count, and its expectation
  mu' d1 d2 n^3 (Sec. 2.2) within 5 sigma;
* identities: Y = I, Y = all ones, zero density, linearity in Y.

``test_planted_mistakes_are_caught`` compiles copies of the oracle with one
plausible mistake each (a dropped term, a wrong sign, a transposed operand,
the literal Case-B "leave the J loop", the floor(mu) upper limit, a wrong
count) and checks that at least one pin fails for every copy.
"""
from __future__ import annotations

import itertools
import math
import os
import re
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import (afmm_case_a, afmm_case_b, classical_ijk, classical_ikj,
                    expected_additions)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53  # unit roundoff of FP64


# ---------------------------------------------------------------- helpers
def load_golden(name):
    blocks, key, case, n, adds = {}, None, None, None, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head = line.split()
            if head[0] == "case":
                case = head[1]
            elif head[0] == "n":
                n = int(head[1])
            elif head[0] == "additions":
                adds = int(head[1])
            elif head[0] in ("X", "Y", "Z"):
                key = head[0]
                blocks[key] = []
            else:
                blocks[key].append([float(v) for v in head])
    return case, n, {k: np.array(v) for k, v in blocks.items()}, adds


def exact_product(X, Y):
    """Z = X * Y in exact rational arithmetic (brute force, tiny n)."""
    n = X.shape[0]
    Xf = [[Fraction(float(X[i, k])) for k in range(n)] for i in range(n)]
    Yf = [[Fraction(float(Y[k, j])) for j in range(n)] for k in range(n)]
    return [[sum((Xf[i][k] * Yf[k][j] for k in range(n)), Fraction(0))
             for j in range(n)] for i in range(n)]


def summation_bound(X, Y, case):
    """Bound on |oracle - exact| per entry for recursive summation.

    Z[i][j] is built by m_ij additions of Base values; the error of a
    recursive sum of m terms is at most gamma_m * sum|terms| with
    gamma_m = m u / (1 - m u).
    """
    R = Y if case == "A" else X
    B = X if case == "A" else Y
    Ab, Ar = np.abs(B.astype(np.float64)), R.astype(np.float64)
    n = X.shape[0]
    if case == "A":
        m = (Ab != 0).astype(np.float64) @ Ar
        s = Ab @ Ar
    else:
        m = Ar @ (Ab != 0).astype(np.float64)
        s = Ar @ Ab
    g = m * U / (1.0 - m * U)
    return g * s + 1e-300


def counter_closed_form(X, Y, case):
    """Additions = sum over (i,k,j) with Base != 0 of the Rep-factor."""
    if case == "A":   # Base = X[i,k], Rep = Y[k,j]
        return int(np.sum(np.count_nonzero(X, axis=0).astype(np.int64)
                          * Y.astype(np.int64).sum(axis=1)))
    # Base = Y[k,j], Rep = X[i,k]
    return int(np.sum(X.astype(np.int64).sum(axis=0)
                      * np.count_nonzero(Y, axis=1).astype(np.int64)))


def run_case(case, X, Y, rows=None):
    return (afmm_case_a if case == "A" else afmm_case_b)(X, Y, rows)


def rand_instance(rng, n, case, real_kind="float", d_real=0.7, d_rep=0.8,
                  rep_max=9):
    rep = rng.integers(0, rep_max + 1, size=(n, n)).astype(np.int64)
    rep[rng.random((n, n)) > d_rep] = 0
    if real_kind == "float":
        real = rng.uniform(-1, 1, size=(n, n))
    elif real_kind == "dyadic":
        real = rng.integers(-4096, 4097, size=(n, n)) / 1024.0
    else:  # integer-valued real factor
        real = rng.integers(-127, 128, size=(n, n)).astype(np.int64)
    real[rng.random((n, n)) > d_real] = 0
    return (real, rep) if case == "A" else (rep, real)


# ---------------------------------------------------------------- pins
def pin_golden():
    for name in ("caseA_3x3_hand.txt", "caseB_2x2_hand.txt",
                 "caseA_identity_4x4_hand.txt"):
        case, n, b, adds = load_golden(name)
        X, Y, Zg = b["X"], b["Y"], b["Z"]
        if case == "A":
            Z, a = afmm_case_a(X, Y.astype(np.int64))
        else:
            Z, a = afmm_case_b(X.astype(np.int64), Y)
        assert Z.shape == (n, n)
        assert np.array_equal(Z, Zg), (name, Z, Zg)
        assert a == adds, (name, a, adds)


def pin_brute_force_exact_integers():
    rng = np.random.default_rng(11)
    for n in range(1, 9):
        for case in "AB":
            X, Y = rand_instance(rng, n, case, real_kind="int")
            Z, a = run_case(case, X, Y)
            E = exact_product(X, Y)
            assert Z.dtype == np.int64
            assert all(int(Z[i, j]) == E[i][j] for i in range(n)
                       for j in range(n)), (case, n)
            assert a == counter_closed_form(X, Y, case)


def pin_exhaustive_2x2():
    """Every 2x2 pair with Base in {-1, 0, 1.5} and Rep in {0, 1, 2}."""
    base_vals, rep_vals = (-1.0, 0.0, 1.5), (0, 1, 2)
    reps = [np.array(v, dtype=np.int64).reshape(2, 2)
            for v in itertools.product(rep_vals, repeat=4)]
    bases = [np.array(v, dtype=np.float64).reshape(2, 2)
             for v in itertools.product(base_vals, repeat=4)]
    for B in bases:
        for R in reps:
            ZA, aA = afmm_case_a(B, R)
            assert np.array_equal(ZA, B @ R.astype(np.float64))
            assert aA == counter_closed_form(B, R, "A")
            ZB, aB = afmm_case_b(R, B)
            assert np.array_equal(ZB, R.astype(np.float64) @ B)
            assert aB == counter_closed_form(R, B, "B")


def pin_fp64_within_summation_bound():
    rng = np.random.default_rng(12)
    for n in (1, 3, 7, 12):
        for case in "AB":
            X, Y = rand_instance(rng, n, case, real_kind="float")
            Z, _ = run_case(case, X, Y)
            E = exact_product(X, Y)
            err = np.array([[abs(Fraction(float(Z[i, j])) - E[i][j])
                             for j in range(n)] for i in range(n)],
                           dtype=np.float64)
            assert np.all(err <= summation_bound(X, Y, case)), (case, n)


def pin_dyadic_bit_exact_vs_library_product():
    """Dyadic Base values: every partial sum is exact, so oracle == X @ Y."""
    rng = np.random.default_rng(13)
    for n in (5, 37, 64, 97):
        for case in "AB":
            X, Y = rand_instance(rng, n, case, real_kind="dyadic")
            Z, a = run_case(case, X, Y)
            ref = X.astype(np.float64) @ Y.astype(np.float64)
            assert np.array_equal(Z, ref), (case, n)
            assert a == counter_closed_form(X, Y, case)


def pin_integer_bit_exact_vs_library_product():
    rng = np.random.default_rng(14)
    for n in (16, 33, 128):
        for case in "AB":
            X, Y = rand_instance(rng, n, case, real_kind="int")
            Z, _ = run_case(case, X, Y)
            assert np.array_equal(Z, X.astype(np.int64) @ Y.astype(np.int64))


def pin_random_fp64_vs_classical():
    rng = np.random.default_rng(15)
    for n in (64, 129):
        for case in "AB":
            X, Y = rand_instance(rng, n, case, real_kind="float")
            Z, _ = run_case(case, X, Y)
            ref = X.astype(np.float64) @ Y.astype(np.float64)
            assert oracle.rel_frobenius_error(Z, ref) < 1e-14
            assert np.all(np.abs(Z - ref) <= 2 * summation_bound(X, Y, case)
                          + 4 * U * np.abs(ref))


def pin_identities():
    rng = np.random.default_rng(16)
    n = 23
    X, _ = rand_instance(rng, n, "A", real_kind="float")
    I = np.eye(n, dtype=np.int64)
    Z, a = afmm_case_a(X, I)                      # Y = I  =>  Z = X
    assert np.array_equal(Z, X) and a == np.count_nonzero(X)
    Z, a = afmm_case_b(I, X)                      # X = I (case B) => Z = Y
    assert np.array_equal(Z, X) and a == np.count_nonzero(X)
    ones = np.ones((n, n), dtype=np.int64)        # Y = 1 => row sums
    Z, a = afmm_case_a(X, ones)
    rs = np.array([math.fsum(r) for r in X])
    assert np.allclose(Z, np.repeat(rs[:, None], n, axis=1), rtol=0,
                       atol=64 * U * np.abs(X).sum(axis=1).max())
    assert a == np.count_nonzero(X) * n
    Z, a = afmm_case_a(np.zeros((n, n)), ones)    # d1 = 0 => Z = 0, no adds
    assert not Z.any() and a == 0
    Z, a = afmm_case_b(np.zeros((n, n), dtype=np.int64), X)
    assert not Z.any() and a == 0
    # Linearity in the Rep-factor: Z(X, Y1 + Y2) = Z(X, Y1) + Z(X, Y2),
    # exact for integer Base values.
    Xi = rng.integers(-50, 51, size=(n, n)).astype(np.int64)
    Y1 = rng.integers(0, 5, size=(n, n)).astype(np.int64)
    Y2 = rng.integers(0, 5, size=(n, n)).astype(np.int64)
    Z12, a12 = afmm_case_a(Xi, Y1 + Y2)
    Z1, a1 = afmm_case_a(Xi, Y1)
    Z2, a2 = afmm_case_a(Xi, Y2)
    assert np.array_equal(Z12, Z1 + Z2) and a12 == a1 + a2


def _count_sigma(n, d1, d2, mu_prime):
    """Std. dev. of the addition count under the iid law used below.

    adds = sum_k c_k s_k with c_k ~ Bin(n, d1) non-zeros in column k of X and
    s_k the sum of row k of Y (n iid entries: non-zero with prob. d2, value
    V = 1 + Poisson(mu' - 1)); the n terms are independent.
    """
    ev2 = (mu_prime - 1.0) + mu_prime ** 2
    ey, ey2 = d2 * mu_prime, d2 * ev2
    ec, vc = n * d1, n * d1 * (1 - d1)
    es, vs = n * ey, n * (ey2 - ey ** 2)
    var_cs = (vc + ec ** 2) * (vs + es ** 2) - (ec * es) ** 2
    return math.sqrt(n * var_cs)


def pin_expected_additions():
    """Counter vs E(A) = mu' d1 d2 n^3 (Sec. 2.2) at Table 1's points."""
    n = 96
    points = [(1, 1 / 3, 1 / 2), (3, 1 / 3, 1 / 2), (5, 1 / 3, 1 / 2),
              (7, 1 / 3, 1 / 2), (14, 1 / 5, 2 / 5), (21, 1 / 5, 2 / 5)]
    for seed, (mu_p, d1, d2) in enumerate(points):
        rng = np.random.default_rng(100 + seed)
        X = rng.uniform(-1, 1, size=(n, n))
        X[rng.random((n, n)) >= d1] = 0.0
        V = 1 + rng.poisson(mu_p - 1, size=(n, n))
        Y = np.where(rng.random((n, n)) < d2, V, 0).astype(np.int64)
        _, a = afmm_case_a(X, Y)
        e = expected_additions(mu_p, d1, d2, n)
        assert abs(a - e) <= 5 * _count_sigma(n, d1, d2, mu_p), (mu_p, a, e)


def pin_classical_loops_agree():
    rng = np.random.default_rng(17)
    X, Y = rand_instance(rng, 41, "A", real_kind="dyadic")
    ref = X @ Y.astype(np.float64)
    assert np.array_equal(classical_ijk(X, Y), ref)
    assert np.array_equal(classical_ikj(X, Y), ref)


PINS = [pin_golden, pin_brute_force_exact_integers, pin_exhaustive_2x2,
        pin_fp64_within_summation_bound,
        pin_dyadic_bit_exact_vs_library_product,
        pin_integer_bit_exact_vs_library_product,
        pin_random_fp64_vs_classical, pin_identities,
        pin_expected_additions, pin_classical_loops_agree]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


# ---------------------------------------------------------------- host logic
def test_rejects_invalid_rep_factors():
    X = np.ones((3, 3))
    with pytest.raises(ValueError):
        afmm_case_a(X, -np.ones((3, 3), dtype=np.int64))
    with pytest.raises(ValueError):
        afmm_case_a(X, np.full((3, 3), 0.5))
    with pytest.raises(ValueError):
        afmm_case_b(np.full((3, 3), 1.5), X)
    with pytest.raises(ValueError):
        afmm_case_a(np.ones((2, 3)), np.ones((2, 3), dtype=np.int64))


def test_row_sample_matches_full_and_thread_count():
    rng = np.random.default_rng(18)
    for case in "AB":
        X, Y = rand_instance(rng, 150, case, real_kind="float")
        Zf, af = run_case(case, X, Y)
        rows = np.array([0, 1, 2, 17, 99, 100, 149])
        Zs, _ = run_case(case, X, Y, rows)
        assert np.array_equal(Zs, Zf[rows])
        t = oracle.oracle_threads()
        oracle.set_oracle_threads(1)
        try:
            Z1, a1 = run_case(case, X, Y)
        finally:
            oracle.set_oracle_threads(t)
        assert np.array_equal(Z1, Zf) and a1 == af


def test_realised_parameters():
    X = np.array([[0.0, 1.0], [2.0, 0.0]])
    Y = np.array([[0, 3], [1, 0]], dtype=np.int64)
    p = oracle.realised_parameters(X, Y, "A")
    assert p == {"d1": 0.5, "d2": 0.5, "mu_prime": 2.0, "mu": 1.0}
    assert expected_additions(2.0, 0.5, 0.5, 2) == 4.0


# ---------------------------------------------------------------- mutants
MUTANTS = [
    # (id, function, text to find, replacement); the loops live in the
    # column-window forms that the plain entry points call.
    ("caseB_literal_leave_J_loop", "afmm_oracle_caseB_f64_cols",
     "if (base == 0.0) continue;", "if (base == 0.0) break;"),
    ("caseA_dropped_last_k", "afmm_oracle_caseA_f64_cols",
     "for (int64_t k = 0; k < n; ++k)", "for (int64_t k = 0; k < n - 1; ++k)"),
    ("caseA_transposed_Y", "afmm_oracle_caseA_f64_cols",
     "Y[k * n + j]", "Y[j * n + k]"),
    ("caseA_floor_mu_upper_limit", "afmm_oracle_caseA_f64_cols",
     "p < rep;", "p < 4;"),
    ("caseB_wrong_sign", "afmm_oracle_caseB_f64_cols",
     "z[j - j0] += base;", "z[j - j0] -= base;"),
    ("caseA_count_off_by_one", "afmm_oracle_caseA_f64_cols",
     "adds += (uint64_t)rep;", "adds += (uint64_t)rep + 1;"),
    ("caseA_int_skip_inverted", "afmm_oracle_caseA_i64_cols",
     "if (base == 0) continue;", "if (base != 0) continue;"),
    ("caseB_int_rep_from_Y", "afmm_oracle_caseB_i64_cols",
     "const int64_t rep = X[i * n + k];", "const int64_t rep = X[k * n + i];"),
]


def _mutate(src, func, old, new):
    start = src.index(func + "(")
    end = src.index("\n}\n", start)
    body = src[start:end]
    assert old in body, (func, old)
    return src[:start] + body.replace(old, new, 1) + src[end:]


@pytest.mark.parametrize("mid,func,old,new", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_are_caught(tmp_path, mid, func, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__),
                            "afmm_oracle.c")).read()
    c = tmp_path / f"{mid}.c"
    c.write_text(_mutate(src, func, old, new))
    so = tmp_path / f"lib{mid}.so"
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", str(so), str(c)],
                   check=True)
    caught = []
    with oracle.use_library(str(so)):
        for pin in PINS:
            try:
                pin()
            except (AssertionError, ValueError):
                caught.append(pin.__name__)
    assert caught, f"no pin caught the planted mistake {mid}"


@pytest.mark.parametrize("case", ["A", "B"])
@pytest.mark.parametrize("integer", [False, True])
def test_column_window_is_the_full_rows_restricted(case, integer):
    """A column window (used to bound the timed CPU samples) forms every
    element exactly as the full rows do, and counts the additions of its own
    columns: sum over k of [Base != 0] * Rep for those j."""
    rng = np.random.default_rng(41)
    n = 29
    real = (rng.integers(-3, 4, (n, n)) if integer else rng.uniform(-1, 1, (n, n)))
    real = real * (rng.random((n, n)) < 0.7)
    rep = rng.integers(0, 4, (n, n))
    X, Y = (real, rep) if case == "A" else (rep, real)
    fn = afmm_case_a if case == "A" else afmm_case_b
    Zf, _ = fn(X, Y, (4, 17))
    Zw, aw = fn(X, Y, (4, 17), cols=(6, 23))
    assert np.array_equal(Zw, Zf[:, 6:23])
    rows = slice(4, 17)
    if case == "A":
        want = int(((X[rows] != 0).astype(np.int64) @ Y[:, 6:23]).sum())
    else:
        want = int((X[rows] @ (Y[:, 6:23] != 0).astype(np.int64)).sum())
    assert aw == want
