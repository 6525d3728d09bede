"""bench.py's reference arm on the host (CPU test): one JSON line with the
metric and unit of the main arm, the oracle timing it describes as its CPU
baseline, and an e2e figure that moves no bytes to or from a GPU."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--workload", "caseA_n256_f64"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("effective TFLOP/s") and d["unit"] == "TFLOP/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 1 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "caseA_n256_f64"
    # The reference line's config is the main line's workload config.
    sys.path.insert(0, ROOT)
    import bench
    import afmm_inputs as W
    want = bench.workload_config("caseA_n256_f64", W.make("caseA_n256_f64"), 1)
    assert d["config"] == json.loads(json.dumps(want))


def test_cpu_baseline_rows_are_whole_thread_blocks():
    """The CPU baseline hands the oracle contiguous blocks of one row per
    oracle thread, so each call runs one parallel region over all cores."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import afmm_inputs as W
    from oracle import oracle_threads
    inst = W.make("caseB_n4096_f32", n=96, seed=3)
    rows, Zr, el, thr = bench.oracle_rows_timed(inst, 0.0, min_rows=2 * min(oracle_threads(), 96))
    assert thr == min(oracle_threads(), 96)
    assert rows.size % thr == 0 and rows.size >= min(2 * thr, 96 - 96 % thr)
    blocks = rows.reshape(-1, thr)
    assert np.all(np.diff(blocks, axis=1) == 1)
    assert np.all(blocks[:, 0] % thr == 0)
    assert Zr.shape == (rows.size, 96)
