"""bench.py's host-side contract, on the CPU: the reference arm (the float64 oracle timed on
the host cores) prints one JSON line with the keys the contract asks for, and the helpers
that label the roofline pick the Res-GCONV kernel the library uses for a matrix and report
stored DRAM traffic only for the source it was captured on."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np

from paper_2406_00809_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-seconds", "0.5"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["higher_is_better"] is False and d["unit"] == "s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    for key in ("workload", "n", "nnz", "hprec", "restart", "rtol"):
        assert key in d["config"], key
    assert d["scaled_by_iterations"] > 0 and d["extrapolated_from_iterations"] > 0


def test_roofline_labels_and_stored_traffic():
    b = load_bench()
    assert b.gconv_kernel_name(I.convdiff2d(16, 100.0)).startswith("k_gconv_row")
    assert b.gconv_kernel_name(I.powerlaw(2048, seed=7)).startswith("k_gconv ")
    # 4(n+1) + 8 nnz + 2 * 16 * 4 n for a float32 hidden block
    n, nnz = 65536, 326656
    assert b.gconv_bytes(n, nnz, 4) == 4 * (n + 1) + 8 * nnz + 2 * 16 * 4 * n
    stored = json.load(open(os.path.join(ROOT, "profiles", "res_gconv_traffic.json")))
    for wl in ("convdiff256", "powerlaw1m"):
        if wl not in stored:
            assert b.stored_traffic(wl) is None
            continue
        expect = stored[wl]["dram_bytes_per_launch"] if stored[wl]["source_hash"] == b.gconv_source_hash() else None
        assert b.stored_traffic(wl) == expect
    assert b.stored_traffic("no_such_workload") is None
    assert np.isfinite(b.load_peaks()[0])
    # the apply's bytes: norm + encoder, L - 1 layers, the decoder-fused last layer
    L, hb = 8, 4
    expect = 16 * n + 16 * n * hb + (L - 1) * b.gconv_bytes(n, nnz, hb) + 4 * (n + 1) + 8 * nnz + 16 * n * hb + 4 * n
    assert b.apply_bytes(n, nnz, L, hb) == expect
