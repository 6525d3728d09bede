"""The seeded input laws (afmm_inputs.py) realise the stated parameters."""
from __future__ import annotations

import math

import numpy as np
import pytest

import afmm_inputs as W
from oracle import realised_parameters


@pytest.mark.parametrize("point", W.TABLE1_POINTS)
def test_table1_points_realise_mu_prime_and_densities(point):
    mu, d1, d2 = point
    n = 400
    inst = W.table1_point(n, mu, d1, d2, seed=3)
    p = realised_parameters(inst.X, inst.Y, "A")
    # Binomial densities and the mean of ~d2 n^2 non-zero Rep-factors:
    # within five standard deviations.
    for got, want in ((p["d1"], d1), (p["d2"], d2)):
        assert abs(got - want) <= 5 * math.sqrt(want * (1 - want) / n ** 2)
    nnz = np.count_nonzero(inst.Y)
    sd = math.sqrt(max(mu - 1.0, 0.0) / nnz)
    assert abs(p["mu_prime"] - mu) <= 5 * sd + 1e-12
    assert inst.Y.min() >= 0 and inst.Y.dtype == np.uint8
    if mu == 1.0:
        assert set(np.unique(inst.Y)) <= {0, 1}


def test_workload_densities():
    for wl, d_x, d_y in (("caseB_n4096_f32", 0.5, None), ("caseA_n8192_e4m3", 0.7, None),
                         ("caseA_n16384_i8", 0.8, 0.6), ("caseB_n4096_sparse", 1 / 16, 1 / 16)):
        n = 256
        inst = W.make(wl, n=n, seed=1)
        p = realised_parameters(inst.X, inst.Y, inst.case)
        want_x = d_x if wl != "caseB_n4096_sparse" else 1 / math.sqrt(n)
        assert abs(p["d1"] - want_x) <= 5 * math.sqrt(want_x * (1 - want_x) / n ** 2), wl
        if d_y is not None:
            want_y = d_y if wl != "caseB_n4096_sparse" else 1 / math.sqrt(n)
            assert abs(p["d2"] - want_y) <= 5 * math.sqrt(want_y * (1 - want_y) / n ** 2), wl


@pytest.mark.parametrize("wl", ["caseA_n256_f64", "caseB_n4096_f32", "caseA_n8192_e4m3",
                                "caseA_n16384_i8", "caseB_n4096_sparse"])
def test_plan_hints_match_the_oracle_parameters(wl):
    """The hints the GPU legs pass (counted in afmm_inputs, no oracle) equal
    the oracle's statement of d1, d2 and mu' (Sec. 2.2)."""
    inst = W.make(wl, n=96, seed=5)
    h = W.density_hints(inst.X, inst.Y, inst.case)
    p = realised_parameters(inst.X, inst.Y, inst.case)
    for k in ("d1", "d2", "mu_prime"):
        assert h[k] == p[k], k
    rep = inst.Y if inst.case == "A" else inst.X
    real = inst.X if inst.case == "A" else inst.Y
    assert h["rep_max"] == float(rep.max())
    assert h["base_max"] == float(np.abs(real.astype(np.float64)).max())
