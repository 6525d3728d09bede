"""Autotuner and dispatch-model trainer for batched AFMM products.

The autotuner times every candidate kernel variant on each instance as
part of a batch (the batched entry point with copies of the instance and a
forced variant, CUDA events, median of repeats, divided by the copies).
Its table is both the yardstick of a dispatch policy (the per-instance
best variant) and the training data of the MLP cost model, which maps
afmm_dispatch_features() of an instance to one predicted log2-time per
variant.  The network is trained on the GPU with the library's own
kernels (afmm_mlp_loss_grad, afmm_mlp_adam) and saved as JSON;
afmm_set_dispatch_model() installs it.

    python -m paper_1308_2400_gb300.tune --count 300 --out model.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time
from typing import Dict, List, Sequence

import numpy as np

from . import afmm as A

# The batched routes the tuner times and the network chooses among: the
# CUDA-core zero-skip form, and the split BF16 tensor-core form with 128 x 256
# or with 128 x 128 output tiles.
VARIANTS = (A.AFMM_VARIANT_SIMT_F32, A.AFMM_VARIANT_TC_BF16X3,
            A.AFMM_VARIANT_TC_BF16X3_N128)
HIDDEN = 32
DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                             "dispatch_mlp.json")


def instance_desc(inst, variant: int = A.AFMM_VARIANT_AUTO) -> "A.afmm_desc":
    """Descriptor of an afmm_inputs.Instance with its measured d1, d2, mu'."""
    X, Y = inst.X, inst.Y
    n2 = float(inst.n) ** 2 if inst.n else 1.0
    rep = Y if inst.case == "A" else X
    nz = np.count_nonzero(rep)
    mu_p = float(rep.sum(dtype=np.float64)) / nz if nz else 0.0
    return A.make_desc(inst.n, inst.case, inst.x_dtype, inst.y_dtype, "f32", "fp32",
                       variant=variant, d1=np.count_nonzero(X) / n2,
                       d2=np.count_nonzero(Y) / n2, mu_prime=mu_p)


def device_operands(inst):
    import torch
    Xs = inst.x_store if inst.x_store is not None else inst.X
    Ys = inst.y_store if inst.y_store is not None else inst.Y
    X = torch.from_numpy(np.ascontiguousarray(Xs)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(Ys)).cuda()
    Z = torch.empty((inst.n, inst.n), dtype=torch.float32, device="cuda")
    return X, Y, Z


def time_batch(descs, Xs, Ys, Zs, reps: int = 5, warmup: int = 2, rounds: int = 3) -> float:
    """Milliseconds per afmm_mul_batched call: `reps` calls back to back
    between two CUDA events (the host's preparation of a call overlaps the
    GPU work of the one before, as in a loop of calls), median of `rounds`."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        A.afmm_mul_batched(descs, Xs, Ys, Zs, st)
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(1, rounds)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(max(1, reps)):
            A.afmm_mul_batched(descs, Xs, Ys, Zs, st)
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / max(1, reps))
    A.afmm_batched_sync(descs, st)
    return statistics.median(ts)


def copies_for(n: int, sms: int = 152, waves: int = 4) -> int:
    """Copies of an n x n instance that give the grouped tensor-core launch
    about `waves` waves of 128 x 256 tiles (1 .. 64)."""
    tiles = -(-n // 128) * -(-n // 256)
    return int(min(64, max(1, -(-waves * sms // tiles))))


def autotune(insts, reps: int = 5) -> np.ndarray:
    """ms[i, v]: the cost of instance i under VARIANTS[v] inside a batch.

    A batch runs its instances in grouped launches, so what an instance
    adds to a batch is its share of a full launch, not the latency of a
    launch of its own (which, for a small instance, is mostly launch and
    ramp-up time).  Each entry is therefore the time of one batched call
    of copies_for(n) copies of the instance (same X and Y, separate Z),
    divided by the number of copies."""
    import torch
    table = np.zeros((len(insts), len(VARIANTS)))
    for i, inst in enumerate(insts):
        X, Y, Z = device_operands(inst)
        r = copies_for(inst.n)
        Zs = [Z] + [torch.empty_like(Z) for _ in range(r - 1)]
        for v, var in enumerate(VARIANTS):
            d = instance_desc(inst, var)
            table[i, v] = time_batch([d] * r, [X] * r, [Y] * r, Zs, reps=reps) / r
        del X, Y, Z, Zs
    return table


def features(insts) -> np.ndarray:
    return np.array([A.afmm_dispatch_features(instance_desc(t)) for t in insts],
                    dtype=np.float64)


def train(feats: np.ndarray, table_ms: np.ndarray, hidden: int = HIDDEN,
          steps: int = 3000, lr: float = 3e-3, seed: int = 0) -> Dict:
    """Fit log2(us) per variant with the library's GPU kernels (Adam)."""
    import torch
    rows, F = feats.shape
    V = table_ms.shape[1]
    mean = feats.mean(axis=0)
    scale = feats.std(axis=0)
    scale[scale < 1e-6] = 1.0
    Xn = (feats - mean) / scale
    T = np.log2(table_ms * 1e3)
    M = np.isfinite(T).astype(np.float64)
    T = np.where(M > 0, T, 0.0)
    shape = A.mlp_shape(F, hidden, V)
    npar = A.afmm_mlp_param_count(shape)
    rng = np.random.default_rng(seed)
    p0 = np.concatenate([
        rng.standard_normal(F * hidden) * math.sqrt(2.0 / F), np.zeros(hidden),
        rng.standard_normal(hidden * hidden) * math.sqrt(2.0 / hidden), np.zeros(hidden),
        rng.standard_normal(hidden * V) * math.sqrt(1.0 / hidden),
        np.full(V, float(T[M > 0].mean()))])
    assert p0.size == npar
    d = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    P, Xd, Td, Md = d(p0), d(Xn), d(T), d(M)
    G = torch.zeros_like(P)
    m1, m2 = torch.zeros_like(P), torch.zeros_like(P)
    work = torch.empty(A.afmm_mlp_work_floats(shape, rows), device="cuda")
    loss = torch.empty(1, device="cuda")
    count = float(M.sum())
    hist = []
    for step in range(1, steps + 1):
        A.afmm_mlp_loss_grad(shape, P, Xd, Td, Md, rows, count, G, work, loss)
        A.afmm_mlp_adam(npar, P, G, m1, m2, lr, 0.9, 0.999, 1e-8, step)
        if step % 500 == 0 or step == 1:
            hist.append((step, float(loss.item())))
    params = P.cpu().numpy().astype(np.float64)
    return {"features": F, "hidden": hidden, "outputs": V,
            "variants": [int(v) for v in VARIANTS], "params": params.tolist(),
            "mean": mean.tolist(), "scale": scale.tolist(),
            "loss_history": hist, "rows": rows}


def predict(model: Dict, feats: np.ndarray) -> np.ndarray:
    """Predicted log2(us) per variant with the library's GPU forward."""
    import torch
    F, H, V = model["features"], model["hidden"], model["outputs"]
    shape = A.mlp_shape(F, H, V)
    Xn = (feats - np.array(model["mean"])) / np.array(model["scale"])
    rows = Xn.shape[0]
    d = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    P = torch.empty((rows, V), device="cuda")
    work = torch.empty(A.afmm_mlp_work_floats(shape, rows), device="cuda")
    A.afmm_mlp_forward(shape, d(model["params"]), d(Xn), rows, P, work)
    return P.cpu().numpy().astype(np.float64)


def install(model: Dict) -> None:
    A.afmm_set_dispatch_model(A.mlp_shape(model["features"], model["hidden"],
                                          model["outputs"]),
                              np.array(model["params"], np.float32),
                              np.array(model["mean"], np.float32),
                              np.array(model["scale"], np.float32),
                              np.array(model["variants"], np.int32))


def load(path: str = DEFAULT_MODEL) -> Dict:
    with open(path) as f:
        return json.load(f)


def regret(table_ms: np.ndarray, choice: Sequence[int]) -> float:
    """sum_i t_i(choice_i) / sum_i min_v t_i(v) - 1 over an autotune table."""
    ch = np.asarray(choice, dtype=np.int64)
    picked = table_ms[np.arange(len(ch)), ch].sum()
    return float(picked / table_ms.min(axis=1).sum() - 1.0)


def route_index(variant: int) -> int:
    """Index into VARIANTS of a batched variant code."""
    return VARIANTS.index(int(variant))


def paper_count_choice(insts, threshold: float) -> List[int]:
    """The method without the network: the paper's addition count
    mu' d1 d2 n^3 (Sec. 2.2) against one fitted threshold -- below it the
    zero-skipping CUDA-core kernel (index 0), above it tensor cores."""
    out = []
    for t in insts:
        d = instance_desc(t)
        adds = max(d.mu_prime, 0.0) * d.d1 * d.d2 * float(t.n) ** 3
        out.append(0 if adds < threshold else 1)
    return out


def fit_paper_threshold(insts, table_ms: np.ndarray) -> float:
    """Threshold on mu'd1d2n^3 minimising the summed time on the table."""
    best, best_t = math.inf, 0.0
    cands = sorted({0.0} | {max(instance_desc(t).mu_prime, 0.0) * instance_desc(t).d1 *
                            instance_desc(t).d2 * float(t.n) ** 3 for t in insts})
    for thr in cands + [math.inf]:
        ch = paper_count_choice(insts, thr)
        tot = table_ms[np.arange(len(ch)), ch].sum()
        if tot < best:
            best, best_t = tot, thr
    return best_t


def main():
    import torch
    import afmm_inputs as W
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--count", type=int, default=300)
    ap.add_argument("--seed", type=int, default=101)
    ap.add_argument("--n-max", type=int, default=2048)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--steps", type=int, default=3000)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    insts = W.batched_mix(count=args.count, seed=args.seed, n_max=args.n_max)
    table = autotune(insts)
    feats = features(insts)
    model = train(feats, table, steps=args.steps)
    pred = predict(model, feats)
    choice = pred.argmin(axis=1)
    model["train_regret"] = regret(table, choice)
    model["train_seconds"] = time.time() - t0
    model["train_set"] = {"law": "batched_512 law", "count": args.count,
                          "seed": args.seed}
    with open(args.out, "w") as f:
        json.dump(model, f)
    best = table.argmin(axis=1)
    print(json.dumps({"regret_train": model["train_regret"],
                      "loss": model["loss_history"][-1],
                      "best_route_share": [float((best == v).mean())
                                           for v in range(len(VARIANTS))],
                      "seconds": model["train_seconds"]}))


if __name__ == "__main__":
    main()
