"""Seeded synthetic inputs for the AFMM product (arXiv 1308.2400).

This module draws the input matrices that both the CPU oracle and the CUDA
library consume.  It holds none of the method's arithmetic: it only draws
values from the stated laws, zeroes entries to reach the stated densities and
stores them in the requested dtypes.

The paper fixes no distribution (Sec. 2: the real factor is "generated
randomly using some probability distribution"; Sec. 2.3.1 gives only d1, d2
and mu').  The five workloads below follow the problem statement (one factor
real, the other non-negative integer Rep-factors; densities d1, d2; mean
mu') with explicit laws:

  caseA_n256_f64     case A, n=256: X FP64 U(-1,1), d1=0.9; Y int32 U{0..9}.
  caseB_n4096_f32    case B, n=4096: X int32 U{0..15}, d1=0.5; Y FP32 N(0,1).
  caseA_n8192_e4m3   case A, n=8192: X FP32 U(-1,1), d1=0.7; Y Poisson(3)
                     clipped to [0,16], stored as FP8 e4m3 (exact).
  caseB_n4096_sparse case B, n=4096, the quadratic regime d1 d2 = 1/n of
                     Sec. 2.2: X int32 U{0..15}, d1 = 1/64; Y FP32 N(0,1),
                     d2 = 1/64.
  caseA_n16384_i8    case A, n=16384: X int8 U[-127,127], d1=0.8;
                     Y int8 U{0..15}, d2=0.6.
  batched_512        512 instances, n log-uniform in [64,2048], d1, d2
                     U[0.05,1], mu in {0.5,1,2,4,8} (Poisson Rep-factors),
                     real factor FP32 N(0,1), cases A/B half and half.
  table1_point       case A at Table 1's points: n 250..2000, (mu', d1, d2)
                     in {1,3,5,7} x (1/3, 1/2) and {14,21} x (1/5, 2/5).

Density reading: values are drawn from the law, then each entry is kept with
probability d / (1 - P(value == 0)) (capped at 1), so the realised fraction
of non-zero entries is d (or the law's own P(value != 0) when that is below
d).  The size n of every workload is a parameter so the same laws serve
small parity cases.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = ["Instance", "WORKLOADS", "make", "batched_mix", "rng_for",
           "encode_e4m3_integers", "table1_point", "TABLE1_POINTS", "TABLE1_SIZES",
           "density_hints"]


@dataclass
class Instance:
    """One AFMM problem: Z = X * Y, n x n, row-major."""
    case: str                      # "A": X real, Y Rep-factors; "B": swapped
    X: np.ndarray
    Y: np.ndarray
    name: str = ""
    # Storage the GPU path reads when it differs from the integer values
    # (e.g. Y as FP8 e4m3 bytes); the oracle always reads X and Y.
    x_store: Optional[np.ndarray] = None
    y_store: Optional[np.ndarray] = None
    x_dtype: str = ""
    y_dtype: str = ""
    z_dtype: str = "f32"
    target: str = "fp32"           # "fp32", "fp64" or "exact"
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])


def density_hints(X: np.ndarray, Y: np.ndarray, case: str) -> dict:
    """Counts of a drawn instance that a caller passes as plan hints.

    d1, d2: fractions of non-zero entries of X and Y; mu_prime: the mean of
    the non-zero entries of the integer factor (Y in case A, X in case B);
    rep_max / base_max: the largest integer entry and the largest |real|
    entry.  Counting only: these are the parameters the paper assumes known
    in advance, read off the arrays this module drew.
    """
    X = np.asarray(X)
    Y = np.asarray(Y)
    n2 = X.size
    rep, real = (Y, X) if case.upper() == "A" else (X, Y)
    nz = int(np.count_nonzero(rep))
    total = float(rep.sum(dtype=np.float64))
    return {"d1": float(np.count_nonzero(X)) / n2 if n2 else 0.0,
            "d2": float(np.count_nonzero(Y)) / n2 if n2 else 0.0,
            "mu_prime": total / nz if nz else 0.0,
            "rep_max": float(rep.max()) if rep.size else 0.0,
            "base_max": float(np.abs(real.astype(np.float64)).max()) if real.size else 0.0}


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for (seed, stream); streams keep X and Y independent."""
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _keep_mask(rng, shape, d: float, p_nonzero: float) -> np.ndarray:
    keep = min(1.0, d / p_nonzero) if p_nonzero > 0 else 1.0
    if keep >= 1.0:
        return np.ones(shape, dtype=bool)
    return rng.random(shape, dtype=np.float32) < np.float32(keep)


def encode_e4m3_integers(v: np.ndarray) -> np.ndarray:
    """Store integers 0..16 as FP8 e4m3 bytes (exact for that range).

    Uses PyTorch's float8_e4m3fn conversion; raises if a value would not be
    exact.
    """
    import torch
    v = np.asarray(v)
    if v.size and (v.min() < 0 or v.max() > 16):
        raise ValueError("e4m3 storage holds integers 0..16 exactly")
    t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32))
    b = t.to(torch.float8_e4m3fn)
    if not torch.equal(b.to(torch.float32), t):
        raise ValueError("value not exact in e4m3")
    return b.view(torch.uint8).numpy().copy()


def _case_a_n256_f64(n: int, seed: int) -> Instance:
    rx, ry, rm = rng_for(seed, 1), rng_for(seed, 2), rng_for(seed, 3)
    X = rx.uniform(-1.0, 1.0, size=(n, n))
    X[~_keep_mask(rm, (n, n), 0.9, 1.0)] = 0.0
    Y = ry.integers(0, 10, size=(n, n), dtype=np.int32)
    return Instance("A", X, Y, name="caseA_f64", x_dtype="f64", y_dtype="i32",
                    z_dtype="f64", target="fp64")


def _case_b_n4096_f32(n: int, seed: int) -> Instance:
    rx, ry, rm = rng_for(seed, 1), rng_for(seed, 2), rng_for(seed, 3)
    X = rx.integers(0, 16, size=(n, n), dtype=np.int32)
    X[~_keep_mask(rm, (n, n), 0.5, 15.0 / 16.0)] = 0
    Y = ry.standard_normal(size=(n, n), dtype=np.float32)
    return Instance("B", X, Y, name="caseB_f32", x_dtype="i32", y_dtype="f32",
                    z_dtype="f32", target="fp32")


def _case_b_n4096_sparse(n: int, seed: int) -> Instance:
    rx, ry, rm1, rm2 = (rng_for(seed, 1), rng_for(seed, 2), rng_for(seed, 3),
                        rng_for(seed, 4))
    d = 1.0 / math.sqrt(max(n, 1))           # d1 = d2 = n^-1/2, d1 d2 = 1/n
    X = rx.integers(0, 16, size=(n, n), dtype=np.int32)
    X[~_keep_mask(rm1, (n, n), d, 15.0 / 16.0)] = 0
    Y = ry.standard_normal(size=(n, n), dtype=np.float32)
    Y[~_keep_mask(rm2, (n, n), d, 1.0)] = 0.0
    return Instance("B", X, Y, name="caseB_sparse", x_dtype="i32", y_dtype="f32",
                    z_dtype="f32", target="fp32")


def _case_a_n8192_e4m3(n: int, seed: int) -> Instance:
    rx, ry, rm = rng_for(seed, 1), rng_for(seed, 2), rng_for(seed, 3)
    X = rx.uniform(-1.0, 1.0, size=(n, n)).astype(np.float32)
    X[~_keep_mask(rm, (n, n), 0.7, 1.0)] = 0.0
    Y = np.minimum(ry.poisson(3.0, size=(n, n)), 16).astype(np.int32)
    inst = Instance("A", X, Y, name="caseA_e4m3", x_dtype="f32",
                    y_dtype="e4m3", z_dtype="f32", target="fp32")
    inst.y_store = encode_e4m3_integers(Y)
    return inst


def _case_a_n16384_i8(n: int, seed: int) -> Instance:
    rx, ry, rm1, rm2 = (rng_for(seed, 1), rng_for(seed, 2), rng_for(seed, 3),
                        rng_for(seed, 4))
    X = rx.integers(-127, 128, size=(n, n), dtype=np.int8)
    X[~_keep_mask(rm1, (n, n), 0.8, 254.0 / 255.0)] = 0
    Y = ry.integers(0, 16, size=(n, n), dtype=np.int8)
    Y[~_keep_mask(rm2, (n, n), 0.6, 15.0 / 16.0)] = 0
    return Instance("A", X, Y, name="caseA_i8", x_dtype="i8", y_dtype="i8",
                    z_dtype="i32", target="exact")


_MAKERS = {
    "caseA_n256_f64": (_case_a_n256_f64, 256),
    "caseB_n4096_f32": (_case_b_n4096_f32, 4096),
    "caseB_n4096_sparse": (_case_b_n4096_sparse, 4096),
    "caseA_n8192_e4m3": (_case_a_n8192_e4m3, 8192),
    "caseA_n16384_i8": (_case_a_n16384_i8, 16384),
}

WORKLOADS = tuple(_MAKERS) + ("batched_512",)


def make(workload: str, n: Optional[int] = None, seed: int = 0) -> Instance:
    """Draw one instance of a named workload, at its own n or at ``n``."""
    fn, n_default = _MAKERS[workload]
    inst = fn(int(n_default if n is None else n), int(seed))
    inst.name = f"{workload}" if n is None else f"{workload}@n={n}"
    return inst


# Table 1's parameter points (Sec. 3): (mu', d1, d2) and the sizes n.
TABLE1_POINTS = ((1.0, 1 / 3, 1 / 2), (3.0, 1 / 3, 1 / 2), (5.0, 1 / 3, 1 / 2),
                 (7.0, 1 / 3, 1 / 2), (14.0, 1 / 5, 2 / 5), (21.0, 1 / 5, 2 / 5))
TABLE1_SIZES = (250, 500, 750, 1000, 1250, 1500, 1750, 2000)


def table1_point(n: int, mu_prime: float, d1: float, d2: float,
                 seed: int = 0) -> Instance:
    """Case A at one of Table 1's parameter points.

    X FP32 U(-1,1) with density d1.  Y Rep-factors (uint8) with density d2
    whose non-zero values are 1 + Poisson(mu' - 1) -- all ones for mu' = 1 --
    so that their mean is mu' (the paper names mu', d1 and d2 only).
    """
    rx, ry, rm1, rm2 = (rng_for(seed, 11), rng_for(seed, 12), rng_for(seed, 13),
                        rng_for(seed, 14))
    X = rx.uniform(-1.0, 1.0, size=(n, n)).astype(np.float32)
    X[~_keep_mask(rm1, (n, n), d1, 1.0)] = 0.0
    if mu_prime > 1.0:
        Y = 1 + ry.poisson(mu_prime - 1.0, size=(n, n))
    else:
        Y = np.ones((n, n), dtype=np.int64)
    Y = np.minimum(Y, 255).astype(np.uint8)
    Y[~_keep_mask(rm2, (n, n), d2, 1.0)] = 0
    return Instance("A", X, Y, name=f"table1[n={n},mu'={mu_prime:g}]", x_dtype="f32",
                    y_dtype="u8", z_dtype="f32", target="fp32",
                    params={"mu_prime": mu_prime, "d1": d1, "d2": d2})


def batched_mix(count: int = 512, seed: int = 0, n_min: int = 64,
                n_max: int = 2048) -> List[Instance]:
    """The uneven batched workload: ``count`` independent instances.

    n log-uniform in [n_min, n_max] (rounded), d1, d2 ~ U[0.05, 1],
    mu ~ uniform on {0.5, 1, 2, 4, 8}; the Rep-factor matrix is Poisson(mu)
    (uint8), the real factor FP32 N(0,1); case A or B with probability 1/2.
    """
    r = rng_for(seed, 100)
    out = []
    for t in range(count):
        n = int(round(math.exp(r.uniform(math.log(n_min), math.log(n_max)))))
        d1, d2 = r.uniform(0.05, 1.0), r.uniform(0.05, 1.0)
        mu = float(r.choice([0.5, 1.0, 2.0, 4.0, 8.0]))
        case = "A" if r.random() < 0.5 else "B"
        ri, rr, rm = rng_for(seed, 1000 + 3 * t), rng_for(seed, 1001 + 3 * t), \
            rng_for(seed, 1002 + 3 * t)
        rep = np.minimum(ri.poisson(mu, size=(n, n)), 255).astype(np.uint8)
        real = rr.standard_normal(size=(n, n), dtype=np.float32)
        if case == "A":
            real[~_keep_mask(rm, (n, n), d1, 1.0)] = 0.0
            rep[~_keep_mask(rm, (n, n), d2, 1.0 - math.exp(-mu))] = 0
            X, Y = real, rep
            xd, yd = "f32", "u8"
        else:
            rep[~_keep_mask(rm, (n, n), d1, 1.0 - math.exp(-mu))] = 0
            real[~_keep_mask(rm, (n, n), d2, 1.0)] = 0.0
            X, Y = rep, real
            xd, yd = "u8", "f32"
        out.append(Instance(case, X, Y, name=f"batched[{t}]", x_dtype=xd,
                            y_dtype=yd, z_dtype="f32", target="fp32",
                            params={"d1": d1, "d2": d2, "mu": mu}))
    return out
