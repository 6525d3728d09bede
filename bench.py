#!/usr/bin/env python3
"""Throughput of the AFMM product on GB300 (one JSON line on stdout).

Workload (default): case A, n = 8192, X FP32 U(-1,1) with density 0.7,
Y Poisson(3) clipped to [0,16] stored as FP8 e4m3; Z FP32 at the FP32
target (relative Frobenius error <= 1e-6 against the FP64 oracle).  One
step = one full product through the C ABI, every conversion included.

Metric: effective TFLOP/s = 2 n^3 / time per product (whole job: summed
over ranks; each rank computes its own independent product, no collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl afmm|reference]
                  [--workload W] [--n N] [--variant V] [--quick] [--shard rows]

Beside the main form the line reports, on the same data, the plain FP32
CUDA-core form (plain_fp32), two BF16 slices (two_slices), the FP8 form
(fp8_slices), two FP16 slices (f16_slices), the split done inside the
product kernel (fused_split) and a
product of two real matrices, X times itself (real_x_real); --quick leaves
them out.  --variant 8 makes that real x real product the main one.

--shard rows splits one product by row blocks over the ranks (Y broadcast
over NCCL each step; "scaling": "strong"); by default every rank computes
its own product.

The reference arm (--impl reference) times the CPU oracle (repeated
addition in FP64, Sec. 2) on the host cores on a bounded row sample of the
same workload, in the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("effective TFLOP/s (2n^3) split-BF16 vs plain FP32 at rel err "
          "<=1e-6; % roofline")
FFMA_PER_SM_PER_CLK = 128          # FP32 lanes per SM (4 SMSPs x 32)
SMS = 152
SM_MAX_MHZ = 2070.0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                "bf16_tflops_sustained": 1700.0}, "fallback"


_REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8,
                "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}


class ClockSampler:
    """SM clock, power and clock-event reasons sampled while the timed
    region runs: NVML queried every ~2 ms from a thread (read-only calls;
    a short region still gets many samples), else nvidia-smi every 20 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None
        self.samples = []          # (sm_mhz, max_mhz, reasons bitmask)
        self.stop_flag = False
        self.source = None
        self.nvml = None
        self.handle = None

    def _nvml_open(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return False
        if lib.nvmlInit_v2() != 0:
            return False
        h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.dev)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        except Exception:
            ok = False
        if not ok:
            # CUDA ordinal -> NVML index through CUDA_VISIBLE_DEVICES when it
            # lists plain indices.
            idx = self.dev
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
            if self.dev < len(vis) and vis[self.dev].strip().isdigit():
                idx = int(vis[self.dev])
            ok = lib.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(h)) == 0
        if not ok:
            lib.nvmlShutdown()
            return False
        self.nvml, self.handle = lib, h
        return True

    def _nvml_loop(self):
        import ctypes
        lib, h = self.nvml, self.handle
        clk, mx = ctypes.c_uint(), ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        get_r = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag:
            if (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 and
                    get_r(h, ctypes.byref(rs)) == 0):
                self.samples.append((float(clk.value), float(mx.value), int(rs.value)))
            time.sleep(0.002)

    def start(self):
        if self._nvml_open():
            self.source = "nvml, every 2 ms"
            self.thread = threading.Thread(target=self._nvml_loop, daemon=True)
            self.thread.start()
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.source = "nvidia-smi, every 20 ms"
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.stop_flag = True
            if self.thread:
                self.thread.join(timeout=2)
            self.nvml.nvmlShutdown()
            return summarise_clocks(self.samples, self.source)
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        samples = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm, mx = float(parts[0]), float(parts[1])
            except ValueError:
                continue
            bits = 0
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    bits |= _REASON_BITS[nm]
            samples.append((sm, mx, bits))
        return summarise_clocks(samples, self.source)


def summarise_clocks(samples, source):
    """Median SM clock, largest max clock and the reasons seen."""
    if not samples:
        return None
    reasons = sorted(nm for nm, b in _REASON_BITS.items()
                     if any(s[2] & b for s in samples))
    return {"sm_mhz": statistics.median(s[0] for s in samples),
            "sm_max_mhz": max(s[1] for s in samples), "samples": len(samples),
            "reasons": reasons, "source": source}


def tensor_peak(peaks, region_s):
    """Measured BF16 dense peak for a kernel timed over region_s seconds:
    the burst figure below one second, the sustained (power-capped) one
    beyond."""
    if region_s < 1.0:
        return peaks.get("bf16_tflops", 1900.0), "bf16 burst"
    return peaks.get("bf16_tflops_sustained", 1700.0), "bf16 sustained"


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(count, rank, ws):
    """Units of rank `rank` when `count` independent units are split over
    `ws` ranks: contiguous, sizes differing by at most one."""
    base, extra = divmod(count, ws)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def row_blocks(n, ws, unit=256):
    """Row blocks [r0, r1) of one n x n product for `ws` ranks: whole
    multiples of `unit` rows (the two-SM tile height) except the last
    block's end, as even as those units allow, covering [0, n) in rank
    order.  Row I of Z needs row I of X and all of Y (Sec. 2.1), so each
    rank multiplies its block of X by the whole Y."""
    units = -(-n // unit) if n > 0 else 0
    out = []
    for r in range(ws):
        lo = shard(units, r, ws)
        r0 = min(n, lo.start * unit)
        r1 = min(n, lo.stop * unit)
        out.append((r0, r1))
    return out


def whole_job_value(units_per_rank, flops_per_unit, max_ms):
    """Whole-job throughput (TFLOP/s): every rank's units over the slowest
    rank's time."""
    return sum(units_per_rank) * flops_per_unit / (max_ms * 1e-3) / 1e12


def make_instance(workload, n):
    import afmm_inputs as W
    return W.make(workload, n=n)


def input_hints(inst):
    """Plan hints (d1, d2, mu', magnitudes) counted off the drawn inputs."""
    import afmm_inputs as W
    return W.density_hints(inst.X, inst.Y, inst.case)


# ---------------------------------------------------------------- oracle legs
# The oracle (test infrastructure) runs only in these helpers: the CPU
# baseline and the accuracy checks of results the GPU already produced.  No
# input of a product comes from here.

def workload_config(workload, inst, ws, real_main=False):
    """The `config` object of both arms' JSON lines: the workload alone
    (its name, size, case, dtypes, realised densities, L2 note, ranks)."""
    h = input_hints(inst)
    n = inst.n
    xb = n * n * inst.X.dtype.itemsize
    zb = n * n * {"f32": 4, "f64": 8, "i32": 4}[inst.z_dtype]
    l2 = (f"inputs larger than L2 (X {xb / 2**20:.0f} MiB, Z {zb / 2**20:.0f} MiB)"
          if max(xb, zb) > 129e6 else
          f"operands fit in L2 (X {xb / 2**20:.1f} MiB, Z {zb / 2**20:.1f} MiB)")
    return {"workload": workload, "n": n,
            "case": "REAL (X X)" if real_main else inst.case,
            "x": inst.x_dtype, "y": inst.x_dtype if real_main else inst.y_dtype,
            "z": inst.z_dtype, "d1": h["d1"], "d2": h["d2"], "mu_prime": h["mu_prime"],
            "l2": l2, "parallelism": f"replicas x{ws}"}


def oracle_rows_timed(inst, budget_s, min_rows=1):
    """CPU baseline: the oracle on contiguous blocks of rows (one row per
    oracle thread, so one parallel region spreads over every host core)
    at random block positions, until ~budget_s seconds have passed.
    Returns (rows, Z rows, seconds, threads)."""
    import numpy as np
    from oracle import afmm_case_a, afmm_case_b, oracle_threads
    fn = afmm_case_a if inst.case == "A" else afmm_case_b
    n = inst.n
    thr = max(1, min(oracle_threads(), n))
    rng = np.random.default_rng(1234)
    order = rng.permutation(n // thr) * thr
    done, rows_out, Z_out = 0, [], []
    t0 = time.perf_counter()
    for r0 in order:
        Zr, _ = fn(inst.X, inst.Y, (int(r0), int(r0) + thr))
        rows_out.append(np.arange(r0, r0 + thr, dtype=np.int64))
        Z_out.append(Zr)
        done += thr
        if time.perf_counter() - t0 >= budget_s and done >= min_rows:
            break
    el = time.perf_counter() - t0
    rows = np.concatenate(rows_out)
    return rows, np.concatenate(Z_out), el, thr


def oracle_product_rows(inst, rows):
    """Rows of the oracle's Z (Sec. 2 loops) for an accuracy check."""
    from oracle import afmm_case_a, afmm_case_b
    return (afmm_case_a if inst.case == "A" else afmm_case_b)(inst.X, inst.Y, rows)[0]


def oracle_classical_rows(X, Y, rows):
    """Rows of the oracle's classical FP64 product X Y (real x real check)."""
    from oracle import classical_ikj
    return classical_ikj(X, Y, rows)


def run_reference(args):
    """The oracle (the CPU AFMM of Sec. 2) on the host cores, in the same
    metric.  Each step computes one element block of Z -- one row per
    oracle thread and a column window (at least 256 wide) sized so that the
    K + W steps take about two minutes -- and the value scales the elements
    to 2n^3."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    import numpy as np
    inst = make_instance(args.workload, args.n)
    n = inst.n
    from oracle import afmm_case_a, afmm_case_b, oracle_threads
    fn = afmm_case_a if inst.case == "A" else afmm_case_b
    thr = min(oracle_threads(), n)
    # Calibrate the column window on one block of 256 columns; windows are
    # at least that wide (narrower ones read Y in short pieces).
    w0 = min(n, 256)
    t0 = time.perf_counter()
    fn(inst.X, inst.Y, (0, thr), cols=(0, w0))
    t_cal = max(time.perf_counter() - t0, 1e-6)
    per_step = 100.0 / max(1, args.steps + args.warmup)
    w = int(w0 * per_step / t_cal) // 32 * 32
    w = max(w0, min(n, w))
    times = []
    for i in range(args.warmup + args.steps):
        r0 = (i * thr) % max(1, n - thr + 1)
        j0 = (i * w) % max(1, n - w + 1)
        t0 = time.perf_counter()
        fn(inst.X, inst.Y, (r0, r0 + thr), cols=(j0, j0 + w))
        el = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(el)
    tot_t = sum(times)
    elems = thr * w * len(times)
    value = 2.0 * n * elems / tot_t / 1e12 if tot_t > 0 else 0.0
    sample = (f"{thr} rows x {w} columns of Z per step (every element its n "
              f"repeated-addition terms, FP64), scaled to 2n^3 per product")
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, inst, ws),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": thr,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def simt_kernel_tag(d1):
    """Which CUDA-core FP32 kernel the library picks for a Base density hint
    d1 (< 0: unknown): the zero-skip kernel below 0.16, else the dense one."""
    return "simt_gemm" if 0.0 <= d1 < 0.16 else "simt_dense_kernel"


def ffma_peak_tflops():
    """Nominal FP32 FFMA rate at the maximum SM clock."""
    return SMS * FFMA_PER_SM_PER_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12


def traffic_from_profile(kernel_tag, workload):
    """Bytes per launch from the committed ncu summary, if it still matches
    the kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}_{workload}.txt")
    if not os.path.exists(path):
        return None
    src = {"simt_gemm": "simt_gemm.cu", "simt_dense_kernel": "simt_dense.cu",
           "tc_gemm": "tc_gemm.cu",
           "tc_gemm_fp8": "tc_gemm.cu", "tc_gemm_real": "tc_gemm.cu",
           "tc_exact2": "tc_gemm.cu", "tc_pair_kernel": "tc_gemm.cu",
           "tc_pair_kernel_x8": "tc_gemm.cu",
           "sparse": "sparse.cu"}.get(kernel_tag)
    vals = {}
    with open(path) as f:
        for ln in f:
            if ":" in ln:
                k, v = ln.split(":", 1)
                vals[k.strip()] = v.strip()
    if src:
        h = hashlib.sha256(open(os.path.join(
            ROOT, "paper_1308_2400_gb300", "csrc", src), "rb").read()).hexdigest()[:16]
        if vals.get("source_sha256_16") != h:
            return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def run_afmm(args):
    import numpy as np
    import torch
    from paper_1308_2400_gb300 import Plan, make_desc
    from paper_1308_2400_gb300.afmm import VARIANT_NAMES

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    peaks, peak_src = load_peaks()

    inst = make_instance(args.workload, args.n)
    n = inst.n
    Xs = inst.x_store if inst.x_store is not None else inst.X
    Ys = inst.y_store if inst.y_store is not None else inst.Y
    X = torch.from_numpy(np.ascontiguousarray(Xs)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(Ys)).cuda()
    Xd, Yd = X, Y
    zt = {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32}[inst.z_dtype]
    Z = torch.empty((n, n), dtype=zt, device="cuda")

    prm = input_hints(inst)

    # Magnitude hints (the paper's "known in advance" parameters extend to
    # the largest Rep-factor and Base value); they size the exact form's
    # K chunks and are checked on the device every call.
    rep_max = prm["rep_max"] if inst.target == "exact" else -1.0
    base_max = prm["base_max"] if inst.target == "exact" else -1.0

    def desc(variant, flags=0):
        return make_desc(n, inst.case, inst.x_dtype, inst.y_dtype,
                         inst.z_dtype, inst.target, variant=variant, flags=flags,
                         d1=prm["d1"], d2=prm["d2"], mu_prime=prm["mu_prime"],
                         rep_max=rep_max, base_max=base_max)

    stream = torch.cuda.Stream()

    def timed(plan, steps, warmup, ops=None):
        """Step time over `steps` calls (no per-kernel events in them, so
        small problems replay their CUDA graph), then the dominant kernel's
        duration from events around it on its stream in a second pass."""
        X, Y = ops if ops is not None else (Xd, Yd)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                plan(X, Y, Z, stream)
            plan.sync(stream)
            c0 = plan.counters()
            barrier(ws)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                plan(X, Y, Z, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier(ws)
            plan.sync(stream)
            c1 = plan.counters()
            plan.enable_kernel_timing(True)
            for _ in range(max(3, min(steps, 50))):
                plan(X, Y, Z, stream)
            plan.sync(stream)
            c2 = plan.counters()
            plan.enable_kernel_timing(False)
        ms = e0.elapsed_time(e1) / steps
        kms = c2["timed_ms"] / max(1, c2["timed_launches"])
        launches = c1["kernel_launches"] - c0["kernel_launches"]
        return ms, kms, launches, c2["main_kernel_ctas"]

    # --variant 8: the real x real form as the main product, the workload's
    # X times itself (no Rep-factor).
    real_main = args.variant == 8
    main_ops = (Xd, Xd) if real_main else None
    plan = Plan(make_desc(n, "REAL", inst.x_dtype, inst.x_dtype, "f32", "fp32", variant=8)
                if real_main else desc(args.variant))
    vname = VARIANT_NAMES.get(plan.info["variant"], "?")
    slices = plan.info["slices"]
    clk = ClockSampler(dev) if rank == 0 else None
    if clk:
        clk.start()
    ms, kms, launches, ctas = timed(plan, args.steps, args.warmup, main_ops)
    clocks = clk.stop() if clk else None
    Z_main = Z.cpu().numpy() if (rank == 0 and ws == 1) else None
    ms_max = max_over_ranks(ws, ms)
    flops = 2.0 * n ** 3
    value = whole_job_value([1] * ws, flops, ms_max)

    # Roofline of the dominant (product) kernel.  Tensor peaks: the burst
    # figure when the timed region is short (the GPU stays near its boost
    # clock), the sustained one for regions of a second or more.
    tc = vname.startswith("tc_")
    region_s = ms * args.steps * 1e-3
    bf16_peak, bf16_src = tensor_peak(peaks, region_s)
    if vname == "sparse":
        # HBM-bound: the product kernel reads the compacted lists (8 bytes per
        # non-zero of X and Y) and writes Z once (4 n^2 bytes).
        nnz = float(np.count_nonzero(inst.X) + np.count_nonzero(inst.Y))
        alg = 8.0 * nnz + 4.0 * n * n
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = alg / (kms * 1e-3) / 1e9
        roof = {"bound": "hbm", "unit": "GB/s", "peak_src": f"HBM copy, {peak_src}",
                "achieved": achieved, "peak": peak, "frac": achieved / peak,
                "traffic": traffic_from_profile("sparse", args.workload),
                "kernel": "sp_mul", "kernel_ms": kms, "ctas": ctas,
                "algorithmic_bytes_per_launch": alg}
    elif vname == "tc_bf16x3x3":
        alg = 6 * flops                    # six slice products
        peak = bf16_peak
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "peak_src": f"{bf16_src}, {peak_src}"}
        tag = "tc_gemm_real"
    elif vname in ("tc_fp8x4", "tc_exact_f8"):
        # E4M3 MMAs: the measured BF16 rate times the nominal FP8/BF16 ratio
        # (four slices of the real factor, or two digits of the integers).
        alg = slices * flops
        peak = 2.0 * bf16_peak
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "peak_src": f"2 x {bf16_src} (nominal fp8/bf16 ratio), {peak_src}"}
        tag = "tc_gemm_fp8" if vname == "tc_fp8x4" else "tc_pair_kernel_x8"
    elif tc:
        alg = (1 if vname == "tc_exact" else slices) * flops
        peak = bf16_peak
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "peak_src": f"{bf16_src}, {peak_src}"}
        # The split forms run on CTA pairs from n = 512 (AFMM_TC_PAIR=0: one CTA).
        pair = (vname in ("tc_bf16x3", "tc_bf16x2", "tc_f16x2") and n >= 512
                and os.environ.get("AFMM_TC_PAIR", "1") != "0")
        tag = "tc_exact2" if vname == "tc_exact" else ("tc_pair_kernel" if pair else "tc_gemm")
    else:
        alg = flops
        peak = ffma_peak_tflops()
        roof = {"bound": "alu", "unit": "TFLOP/s",
                "peak_src": f"FP32 FFMA {SMS} SMs x 128 lanes x 2 x {SM_MAX_MHZ:.0f} MHz"}
        # The FP64-target and exact CUDA-core forms run int8 dot products.
        tag = (simt_kernel_tag(prm["d1"]) if vname == "simt_f32" else "simt_dp4a")
    if vname != "sparse":
        achieved = alg / (kms * 1e-3) / 1e12
        roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak,
                     "traffic": traffic_from_profile(tag, args.workload),
                     "kernel": tag, "kernel_ms": kms, "ctas": ctas,
                     "algorithmic_flops_per_launch": alg})
    roof["timed_region_s"] = region_s

    # Plain FP32 CUDA-core form on the same data, when the main form differs.
    plain = None
    if rank == 0 and vname != "simt_f32" and inst.target == "fp32" and not args.quick:
        p2 = Plan(desc(0))
        ms2, kms2, _, _ = timed(p2, max(2, min(args.steps // 4, 100)), 3)
        plain = {"variant": "simt_f32", "value": flops / (ms2 * 1e-3) / 1e12,
                 "ms_per_step": ms2, "kernel_ms": kms2,
                 "kernel": simt_kernel_tag(prm["d1"]),
                 "kernel_frac_of_ffma_peak": flops / (kms2 * 1e-3) / 1e12 / ffma_peak_tflops()}
        p2.close()

    # The split of the real factor done inside the product kernel instead of
    # in a separate pass (Case A), for comparison.
    fused = None
    if rank == 0 and vname == "tc_bf16x3" and inst.case == "A" and not args.quick:
        from paper_1308_2400_gb300.afmm import AFMM_FLAG_FUSED_SPLIT
        p3 = Plan(desc(args.variant, AFMM_FLAG_FUSED_SPLIT))
        ms3, kms3, _, _ = timed(p3, max(2, min(args.steps // 4, 100)), 3)
        fused = {"value": flops / (ms3 * 1e-3) / 1e12, "ms_per_step": ms3,
                 "kernel_ms": kms3}
        p3.close()

    # Two BF16 slices instead of three on the same data: faster, but short of
    # the FP32 target (its error is taken on the CPU-baseline rows below).
    two = None
    Z_two = None
    if rank == 0 and vname == "tc_bf16x3" and not args.quick:
        p4 = Plan(desc(2))
        ms4, kms4, _, _ = timed(p4, max(2, min(args.steps // 4, 100)), 3)
        two = {"variant": "tc_bf16x2", "value": flops / (ms4 * 1e-3) / 1e12,
               "ms_per_step": ms4, "kernel_ms": kms4}
        Z_two = Z.cpu().numpy() if ws == 1 else None
        p4.close()

    # The FP8 form on the same data: four E4M3 slices on the kind::f8f6f4
    # tensor path (twice the BF16 rate); its error is taken below too.
    f8 = None
    Z_f8 = None
    if rank == 0 and vname == "tc_bf16x3" and not args.quick:
        p5 = Plan(desc(7))
        ms5, kms5, _, _ = timed(p5, max(2, min(args.steps // 4, 100)), 3)
        f8_peak = 2.0 * tensor_peak(peaks, ms5 * max(2, min(args.steps // 4, 100)) * 1e-3)[0]
        f8_tf = 4 * flops / (kms5 * 1e-3) / 1e12
        f8 = {"variant": "tc_fp8x4", "value": flops / (ms5 * 1e-3) / 1e12,
              "ms_per_step": ms5, "kernel_ms": kms5, "tensor_tflops": f8_tf,
              "peak": f8_peak, "frac": f8_tf / f8_peak,
              "peak_src": f"2 x bf16 measured (nominal fp8/bf16 ratio), {peak_src}"}
        Z_f8 = Z.cpu().numpy() if ws == 1 else None
        p5.close()

    # The FP16 two-slice form on the same data: the real factor as two
    # row-scaled FP16 slices (Case B: Y's columns), two MMAs per K step at
    # the BF16 rate; its error below.
    h16 = None
    Z_h16 = None
    if rank == 0 and vname == "tc_bf16x3" and not args.quick:
        p7 = Plan(desc(10))
        k7 = max(2, min(args.steps // 4, 100))
        ms7, kms7, _, _ = timed(p7, k7, 3)
        tf7 = 2 * flops / (kms7 * 1e-3) / 1e12
        pk7 = tensor_peak(peaks, ms7 * k7 * 1e-3)
        h16 = {"variant": "tc_f16x2", "value": flops / (ms7 * 1e-3) / 1e12,
               "ms_per_step": ms7, "kernel_ms": kms7, "tensor_tflops": tf7,
               "peak": pk7[0], "frac": tf7 / pk7[0],
               "peak_src": f"{pk7[1]} (FP16 and BF16 share the rate), {peak_src}"}
        Z_h16 = Z.cpu().numpy() if ws == 1 else None
        p7.close()

    # A product of two real matrices (no Rep-factor) with the workload's X as
    # both factors: both split into three BF16 slices, six slice products.
    rr = None
    Z_rr = None
    if rank == 0 and vname == "tc_bf16x3" and inst.case == "A" and not args.quick:
        p6 = Plan(make_desc(n, "REAL", inst.x_dtype, inst.x_dtype, "f32", "fp32"))
        ms6, kms6, _, _ = timed(p6, max(2, min(args.steps // 8, 50)), 3, (Xd, Xd))
        tf6 = 6 * flops / (kms6 * 1e-3) / 1e12
        rr = {"variant": VARIANT_NAMES.get(p6.info["variant"], "?"), "operands": "X, X",
              "value": flops / (ms6 * 1e-3) / 1e12, "ms_per_step": ms6,
              "kernel_ms": kms6, "tensor_tflops": tf6,
              "frac": tf6 / tensor_peak(peaks, ms6 * max(2, min(args.steps // 8, 50)) * 1e-3)[0]}
        Z_rr = Z.cpu().numpy() if ws == 1 else None
        p6.close()

    # End to end through the C ABI with pinned host buffers: copies in,
    # product, copy out, every step.
    e2e = None
    if not args.quick:
        Xh = torch.from_numpy(np.ascontiguousarray(Xs)).pin_memory()
        Yh = Xh if real_main else torch.from_numpy(np.ascontiguousarray(Ys)).pin_memory()
        Zh = torch.empty((n, n), dtype=zt).pin_memory()
        ph = Plan(make_desc(n, "REAL", inst.x_dtype, inst.x_dtype, "f32", "fp32", variant=8)
                  if real_main else desc(args.variant))
        with torch.cuda.stream(stream):
            for _ in range(2):
                ph(Xh, Yh, Zh, stream)
            barrier(ws)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ksteps = max(2, min(args.steps // 4, 100))
            for _ in range(ksteps):
                ph(Xh, Yh, Zh, stream)
            torch.cuda.synchronize()
            t_e2e = (time.perf_counter() - t0) / ksteps
        t_e2e = max_over_ranks(ws, t_e2e)
        e2e = {"value": ws * flops / t_e2e / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(Xh.nbytes + (0 if real_main else Yh.nbytes)),
               "d2h_bytes_per_step": int(Zh.nbytes), "ms_per_step": 1e3 * t_e2e}
        ph.close()

    # CPU baseline: the oracle on a bounded row sample, rank 0 at N = 1;
    # the same rows give the accuracy check of the GPU result.
    cpu = None
    acc = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rows, Zr, el, thr = oracle_rows_timed(inst, args.cpu_seconds)
        cpu = {"value": 2.0 * n * n * rows.size / el / 1e12, "unit": "TFLOP/s",
               "cores": thr, "kind": "oracle",
               "sample": f"{rows.size} of {n} rows of Z, repeated addition in "
                         f"FP64 (Sec. 2 loops), {el:.1f} s; scaled to 2n^3"}
        Zg = Z_main[rows].astype(np.float64)
        num = float(np.linalg.norm(Zg - Zr))
        den = float(np.linalg.norm(Zr))
        acc = {"rel_fro_err_vs_oracle": num / den if den else 0.0,
               "rows_checked": int(rows.size)}
        if real_main:
            r16 = rows[:16]
            Rr = oracle_classical_rows(inst.X, inst.X, r16)
            acc = {"rel_fro_err_vs_oracle": float(
                np.linalg.norm(Z_main[r16].astype(np.float64) - Rr) / np.linalg.norm(Rr)),
                "rows_checked": int(r16.size), "oracle": "classical FP64 product X X"}
        if two is not None and Z_two is not None:
            d2 = float(np.linalg.norm(Z_two[rows].astype(np.float64) - Zr))
            two["rel_fro_err_vs_oracle"] = d2 / den if den else 0.0
        if f8 is not None and Z_f8 is not None:
            d8 = float(np.linalg.norm(Z_f8[rows].astype(np.float64) - Zr))
            f8["rel_fro_err_vs_oracle"] = d8 / den if den else 0.0
        if h16 is not None and Z_h16 is not None:
            dh = float(np.linalg.norm(Z_h16[rows].astype(np.float64) - Zr))
            h16["rel_fro_err_vs_oracle"] = dh / den if den else 0.0
        if rr is not None and Z_rr is not None:
            r16 = rows[:16]
            Rr = oracle_classical_rows(inst.X, inst.X, r16)
            rr["rel_fro_err_vs_oracle"] = float(
                np.linalg.norm(Z_rr[r16].astype(np.float64) - Rr) / np.linalg.norm(Rr))
            rr["rows_checked"] = int(r16.size)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ({"tc_fp8x4": "e4m3", "tc_f16x2": "f16",
                       "tc_exact_f8": "e4m3"}.get(vname, "bf16")) if tc else
                     ("f64" if inst.target == "fp64" else
                                        ("i8" if inst.target == "exact" else "f32")),
            "data": "synthetic",
            "config": workload_config(args.workload, inst, ws, real_main),
            "variant": vname, "slices": slices,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches) * ws, "clocks": clocks,
            "accuracy": acc, "plain_fp32": plain, "fused_split": fused,
            "two_slices": two, "fp8_slices": f8, "f16_slices": h16, "real_x_real": rr,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_shard_rows(args):
    """One product split by row blocks over the ranks (Sec. 2.1: row I of Z
    needs row I of X and all of Y).  Rank r holds rows row_blocks(n, N)[r]
    of X and Z; each step rank 0 broadcasts Y over NCCL and every rank
    multiplies its rows through afmm_mul_rows.  value = 2 n^3 over the
    slowest rank's step ("strong": one product whatever N)."""
    import numpy as np
    import torch
    from paper_1308_2400_gb300 import Plan, make_desc
    from paper_1308_2400_gb300.afmm import VARIANT_NAMES, afmm_mul_rows
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    inst = make_instance(args.workload, args.n)
    n = inst.n
    r0, r1 = row_blocks(n, ws)[rank]
    Xs = inst.x_store if inst.x_store is not None else inst.X
    Ys = inst.y_store if inst.y_store is not None else inst.Y
    Xd = torch.from_numpy(np.ascontiguousarray(Xs[r0:r1])).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Ys)).cuda()
    if rank != 0:
        Yd.zero_()                     # filled by the broadcast of each step
    zt = {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32}[inst.z_dtype]
    Zd = torch.empty((max(r1 - r0, 1), n), dtype=zt, device="cuda")
    h = input_hints(inst)
    plan = Plan(make_desc(n, inst.case, inst.x_dtype, inst.y_dtype, inst.z_dtype,
                          inst.target, variant=args.variant, d1=h["d1"], d2=h["d2"],
                          mu_prime=h["mu_prime"]))
    vname = VARIANT_NAMES.get(plan.info["variant"], "?")
    stream = torch.cuda.current_stream()

    def step():
        if ws > 1:
            dist.broadcast(Yd, src=0)
        afmm_mul_rows(plan, r0, r1, Xd, Yd, Zd, stream)

    for _ in range(args.warmup):
        step()
    plan.sync(stream)
    barrier(ws)
    torch.cuda.synchronize()
    clk = ClockSampler(dev) if rank == 0 else None
    if clk:
        clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop() if clk else None
    plan.sync(stream)
    ms = max_over_ranks(ws, e0.elapsed_time(e1) / args.steps)
    value = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
    acc = None
    if rank == 0 and not args.no_cpu_baseline and r1 > r0:
        rows = np.arange(r0, r1, max(1, (r1 - r0) // 8))
        R = oracle_product_rows(inst, rows)
        Zg = Zd.cpu().numpy()[rows - r0].astype(np.float64)
        acc = {"rel_fro_err_vs_oracle": float(np.linalg.norm(Zg - R) / np.linalg.norm(R)),
               "rows_checked": int(rows.size)}
    if rank == 0:
        cfg = workload_config(args.workload, inst, ws)
        cfg["parallelism"] = f"row blocks x{ws} (Y broadcast each step)"
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic", "config": cfg, "variant": vname,
            "shard": "rows", "rows_per_rank": [b - a for a, b in row_blocks(n, ws)],
            "accuracy": acc, "clocks": clocks}), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """The uneven batched workload: 512 independent instances in one
    afmm_mul_batched call per step (grouped launches in a CUDA graph), the
    variant of each instance picked by the learned dispatcher; beside it the
    autotuner's per-instance best, fixed routes and the paper's count rule."""
    import numpy as np
    import torch
    import afmm_inputs as W
    from paper_1308_2400_gb300 import afmm as A
    from paper_1308_2400_gb300 import tune

    torch.cuda.set_device(0)
    peaks, peak_src = load_peaks()
    insts = W.batched_mix(count=args.count, seed=0)
    ops = [tune.device_operands(t) for t in insts]
    Xs, Ys, Zs = [o[0] for o in ops], [o[1] for o in ops], [o[2] for o in ops]
    flops = float(sum(2.0 * t.n ** 3 for t in insts))
    model = None
    if os.path.exists(tune.DEFAULT_MODEL):
        model = tune.load(tune.DEFAULT_MODEL)
        tune.install(model)
    auto = [tune.instance_desc(t) for t in insts]
    routes_mlp = [tune.route_index(A.afmm_dispatch_variant(d)) for d in auto]

    def forced(routes):
        return [tune.instance_desc(t, tune.VARIANTS[r]) for t, r in zip(insts, routes)]

    clk = ClockSampler(0)
    clk.start()
    ms = tune.time_batch(auto, Xs, Ys, Zs, reps=args.steps, warmup=args.warmup, rounds=1)
    clocks = clk.stop()
    # accuracy of the timed results on a sample of instances
    errs = []
    for i in range(0, len(insts), max(1, len(insts) // 12)):
        t = insts[i]
        rows = np.arange(0, t.n, max(1, t.n // 16))
        R = oracle_product_rows(t, rows)
        Zg = Zs[i].cpu().numpy()[rows].astype(np.float64)
        errs.append(float(np.linalg.norm(Zg - R) / max(np.linalg.norm(R), 1e-300)))
    dispatch = None
    if not args.quick:
        table = tune.autotune(insts, reps=3)
        best = [int(v) for v in table.argmin(axis=1)]
        thr = tune.fit_paper_threshold(insts, table)
        A.afmm_set_dispatch_model(None, None, None, None, None)
        routes_rule = [tune.route_index(A.afmm_dispatch_variant(d)) for d in auto]
        if model is not None:
            tune.install(model)
        policies = {"autotune_best": best, "learned": routes_mlp, "rule": routes_rule,
                    "paper_count_rule": tune.paper_count_choice(insts, thr),
                    "all_tc": [1] * len(insts), "all_tc_n128": [2] * len(insts),
                    "all_simt": [0] * len(insts)}
        # Timed in rounds, each policy once per round in turn, so that a
        # drift of the clock over the run is shared by all of them.
        samples = {name: [] for name in policies}
        rounds = max(2, min(args.steps, 8))
        for _ in range(rounds):
            for name, r in policies.items():
                reps = 3 if name != "all_simt" else 1
                samples[name].append(tune.time_batch(forced(r), Xs, Ys, Zs, reps=reps,
                                                     warmup=1, rounds=1))
        times = {name: statistics.median(v) for name, v in samples.items()}
        no_mlp = {k: v for k, v in times.items() if k not in ("learned", "autotune_best")}
        best_no_mlp = min(no_mlp, key=no_mlp.get)
        dispatch = {
            "batch_ms": times,
            "rounds": rounds,
            "regret_batch": times["learned"] / times["autotune_best"] - 1.0,
            "regret_table": tune.regret(table, routes_mlp),
            "best_no_mlp_policy": best_no_mlp,
            "gain_vs_best_no_mlp": times[best_no_mlp] / times["learned"],
            "gain_vs_paper_count_rule": times["paper_count_rule"] / times["learned"],
            "gain_vs_rule": times["rule"] / times["learned"],
            "paper_count_threshold": thr,
            "autotune_route_share": [float(np.mean(np.asarray(best) == v))
                                     for v in range(len(tune.VARIANTS))],
            "learned_route_share": [float(np.mean(np.asarray(routes_mlp) == v))
                                    for v in range(len(tune.VARIANTS))],
        }
    line = {
        "metric": METRIC, "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "batched_512", "count": len(insts),
                   "sum_2n3": flops, "tc_instances": int(sum(1 for r in routes_mlp if r > 0)),
                   "dispatch": "learned" if model else "rule"},
        "roofline": {"bound": "tensor", "unit": "TFLOP/s",
                     "achieved": 3 * flops / (ms * 1e-3) / 1e12,
                     "peak": tensor_peak(peaks, ms * args.steps * 1e-3)[0],
                     "peak_src": f"{tensor_peak(peaks, ms * args.steps * 1e-3)[1]}, {peak_src}",
                     "frac": 3 * flops / (ms * 1e-3) / 1e12 /
                             tensor_peak(peaks, ms * args.steps * 1e-3)[0],
                     "note": "whole step (conversions + grouped products), 3 slices"},
        "dispatch": dispatch,
        "accuracy": {"max_rel_fro_err_sampled": max(errs), "instances": len(errs)},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


# Table 1 of the paper (Sec. 3): mean seconds on a 1.6 GHz Pentium for the
# classical ikj loop and AFMM at mu' = 1, 3, 5, 7 (d1 = 1/3, d2 = 1/2) and
# 14, 21 (d1 = 1/5, d2 = 2/5).  Context only: other hardware and precision.
TABLE1_SECONDS = {
    250: (0.328, 0.1752, 0.2784, 0.3316, 0.3498, 0.3188, 0.2874),
    500: (2.32, 0.918, 1.5406, 1.943, 2.331, 1.9122, 1.9874),
    750: (7.75533, 2.8475, 4.9718, 6.38, 7.6826, 6.3218, 6.4328),
    1000: (18.43233, 6.67175, 11.8064, 15.073, 18.2756, 14.9158, 15.3374),
    1250: (35.75, 13.0897, 23.0705, 29.489, 35.594, 29.172, 29.9267),
    1500: (61.688, 22.5625, 40.078, 50.9295, 61.718, 50.3515, 52.2),
    1750: (98.515, 36.0235, 63.2655, 80.6235, 97.6955, 80.281, 81.9335),
    2000: (147.078, 53.375, 94.6875, 120.8515, 145.8985, 119.516, 122.491),
}


def run_table1(args):
    """The paper's own parameter grid (Table 1: n = 250..2000, six (mu', d1,
    d2) points), Case A, FP32 target, planner's choice of variant: GPU time
    per product beside the paper's CPU times, which are context only."""
    import numpy as np
    import torch
    import afmm_inputs as W
    from paper_1308_2400_gb300 import Plan, make_desc
    from paper_1308_2400_gb300.afmm import VARIANT_NAMES
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rows_out, worst = [], 0.0
    clk = ClockSampler(0)
    clk.start()
    for n in W.TABLE1_SIZES:
        for j, (mu, d1, d2) in enumerate(W.TABLE1_POINTS):
            inst = W.table1_point(n, mu, d1, d2, seed=n)
            prm = W.density_hints(inst.X, inst.Y, "A")
            X = torch.from_numpy(inst.X).cuda()
            Y = torch.from_numpy(inst.Y).cuda()
            Z = torch.empty((n, n), dtype=torch.float32, device="cuda")
            plan = Plan(make_desc(n, "A", "f32", "u8", "f32", "fp32", d1=prm["d1"],
                                  d2=prm["d2"], mu_prime=prm["mu_prime"]))
            with torch.cuda.stream(stream):
                for _ in range(max(3, args.warmup)):
                    plan(X, Y, Z, stream)
                plan.sync(stream)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    plan(X, Y, Z, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                plan.sync(stream)
            ms = e0.elapsed_time(e1) / args.steps
            r = np.arange(0, n, max(1, n // 8))
            R = oracle_product_rows(inst, r)
            err = float(np.linalg.norm(Z.cpu().numpy()[r] - R) / np.linalg.norm(R))
            worst = max(worst, err)
            paper = TABLE1_SECONDS[n]
            rows_out.append({
                "n": n, "mu_prime": mu, "d1": round(d1, 4), "d2": round(d2, 4),
                "variant": VARIANT_NAMES.get(plan.info["variant"], "?"),
                "gpu_ms": ms, "gpu_tflops_2n3": 2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                "additions_mu_d1_d2_n3": mu * d1 * d2 * n ** 3,
                "paper_afmm_s": paper[1 + j], "paper_ikj_s": paper[0],
                "rel_fro_err_rows": err})
            plan.close()
    clocks = clk.stop()
    tot = sum(r["gpu_ms"] for r in rows_out)
    line = {"metric": "Table 1 grid: GPU ms per product (FP32 target)",
            "value": tot / len(rows_out), "unit": "ms (mean over the grid)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "table1_sweep", "points": len(rows_out)},
            "max_rel_fro_err": worst, "clocks": clocks, "table": rows_out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="afmm", choices=["afmm", "reference"])
    ap.add_argument("--workload", default="caseA_n8192_e4m3")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="skip the plain-FP32 and end-to-end legs")
    ap.add_argument("--count", type=int, default=512,
                    help="instances of the batched workload")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "rows"],
                    help="rows: split one product by row blocks over the ranks")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_512":
        return run_batched(args)
    if args.workload == "table1_sweep":
        return run_table1(args)
    if args.shard == "rows":
        return run_shard_rows(args)
    return run_afmm(args)


if __name__ == "__main__":
    sys.exit(main())
