"""Shared helpers of the test suite: run an instance through the C ABI and
compare it with the oracle."""
from __future__ import annotations

import math

import numpy as np

U32 = 2.0 ** -24   # unit roundoff of FP32
U64 = 2.0 ** -53   # unit roundoff of FP64

# Tolerances the product must meet against the FP64 oracle (relative
# Frobenius error): FP32 target 1e-6, FP64 target 1e-12; integers exact.
FP32_REL_FRO = 1e-6
FP64_REL_FRO = 1e-12


def torch_of(arr, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).to(device)


def gpu_operands(inst):
    """Device tensors for X and Y in the storage the instance declares."""
    X = inst.x_store if inst.x_store is not None else inst.X
    Y = inst.y_store if inst.y_store is not None else inst.Y
    return torch_of(X), torch_of(Y)


def z_torch_dtype(z):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32}[z]


def desc_for(inst, variant=-1, flags=0, hints=True, d1_hint=None):
    """Descriptor of ``inst``; ``d1_hint`` overrides the X density hint
    (hints steer kernel choice only, never the result)."""
    from afmm_inputs import density_hints
    from paper_1308_2400_gb300 import make_desc
    d1 = d2 = mp = -1.0
    if hints:
        p = density_hints(inst.X, inst.Y, inst.case)
        d1, d2, mp = p["d1"], p["d2"], p["mu_prime"]
    if d1_hint is not None:
        d1 = d1_hint
    return make_desc(inst.n, inst.case, inst.x_dtype, inst.y_dtype,
                     inst.z_dtype, inst.target, variant=variant, flags=flags,
                     d1=d1, d2=d2, mu_prime=mp)


def run_gpu(inst, variant=-1, flags=0, hints=True, d1_hint=None):
    """Z on the GPU through the C ABI; returns (Z numpy, plan info)."""
    import torch
    from paper_1308_2400_gb300 import Plan
    X, Y = gpu_operands(inst)
    Z = torch.full((inst.n, inst.n), float("nan") if inst.z_dtype != "i32"
                   else -7, dtype=z_torch_dtype(inst.z_dtype), device="cuda")
    plan = Plan(desc_for(inst, variant, flags, hints, d1_hint))
    plan(X, Y, Z)
    plan.sync()
    info = plan.info
    plan.close()
    return Z.cpu().numpy(), info


def oracle_rows(inst, rows=None):
    from oracle import afmm_case_a, afmm_case_b
    fn = afmm_case_a if inst.case == "A" else afmm_case_b
    Z, adds = fn(inst.X, inst.Y, rows)
    return Z


def abs_product(inst, rows=None):
    """(|X| |Y|) restricted to the selected rows, in FP64."""
    Xa = np.abs(inst.X.astype(np.float64))
    if rows is not None:
        Xa = Xa[rows]
    return Xa @ np.abs(inst.Y.astype(np.float64))


def rel_fro(Z, R):
    Z = np.asarray(Z, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    den = math.sqrt(float(np.sum(R * R)))
    num = math.sqrt(float(np.sum((Z - R) ** 2)))
    return num / den if den else (0.0 if num == 0 else math.inf)


def sample_rows(n, count, seed=0):
    """Rows to check at full size: first, last and a seeded spread."""
    rng = np.random.default_rng(seed + n)
    rows = set([0, n - 1]) | set(rng.choice(n, size=min(count, n),
                                            replace=False).tolist())
    return np.array(sorted(rows), dtype=np.int64)
