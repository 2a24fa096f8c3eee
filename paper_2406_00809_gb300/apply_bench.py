"""GNP-apply throughput (HBM GB/s) and the Res-GCONV layer kernel in isolation.

    python -m paper_2406_00809_gb300.apply_bench [--workload powerlaw1m] [--reps 20]
        [--hprec fp32|bf16|both] [--iters 50]

For each hidden-block precision: the whole apply z = M(v) is timed with CUDA events
(L2 flushed by a 256 MB write before every rep, or warm with --warm) and converted to GB/s with the
algorithmic bytes of its kernels; then an FGMRES run of a fixed number of iterations
times every Res-GCONV launch with CUDA events (gnp_profile_gconv).  Prints one JSON
line per precision.  Inputs are synthetic (paper_2406_00809_gb300.inputs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_00809_gb300 import inputs as I  # noqa: E402


def apply_bytes(n, nnz, L, hb):
    """Algorithmic bytes of one apply: norm pass (8n), encoder (8n in, 16 n hb out),
    L-1 layers (CSR 4(n+1) + 8 nnz, hidden in + out), last layer with the decoder
    (CSR, hidden in, 4n out)."""
    csr = 4 * (n + 1) + 8 * nnz
    layer = csr + 2 * n * 16 * hb
    last = csr + n * 16 * hb + 4 * n
    return 8 * n + 8 * n + 16 * n * hb + (L - 1) * layer + last, layer


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="powerlaw1m", choices=["powerlaw1m", "convdiff256", "powerlaw64k"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--hprec", default="both", choices=["fp32", "bf16", "both"])
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--L", type=int, default=8)
    ap.add_argument("--warm", action="store_true", help="no L2 flush between reps")
    a = ap.parse_args()
    import torch
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp
    t0 = time.perf_counter()
    A, _ = I.workload(a.workload)
    gen_s = time.perf_counter() - t0
    n, nnz, L = A.n, A.nnz, a.L
    stream = torch.cuda.Stream()
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    with torch.cuda.stream(stream):
        Mt = gnp.mat_from_csr(A)
        M = gnp.gnp_create(Mt, gnp.make_config(L=L), I.init_weights(L, seed=0))
        v = torch.from_numpy(I.gaussian(n, seed=1)).cuda()
        z = torch.empty(n, dtype=torch.float32, device="cuda")
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        b = torch.from_numpy(I.spmv(A, I.gaussian(n, seed=0))).cuda()
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        precs = ["fp32", "bf16"] if a.hprec == "both" else [a.hprec]
        for p in precs:
            gnp.gnp_set_hprec(M, gnp.H_BF16 if p == "bf16" else gnp.H_FP32)
            hb = 2 if p == "bf16" else 4
            for _ in range(3):
                gnp.gnp_apply(M, v, z, stream=stream)
            times = []
            for _ in range(a.reps):
                if not a.warm:
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                gnp.gnp_apply(M, v, z, stream=stream)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
            tot, layer = apply_bytes(n, nnz, L, hb)
            t_apply = statistics.median(times)
            gnp.gnp_profile_gconv(True)
            x.zero_()
            info = gnp.fgmres_solve(Mt, b, x, M, restart=min(50, a.iters), rtol=1e-30, maxiters=a.iters,
                                    stream=stream, history=False)
            gnp.gnp_profile_gconv(False)
            g_us = info.gconv_ms / info.gconv_launches * 1e3 if info.gconv_launches else None
            # plain layers move `layer` bytes; the decoder-fused last layer fewer
            last = layer - n * 16 * hb + 4 * n
            avg_bytes = ((L - 1) * layer + last) / L
            g_gbs = avg_bytes / (g_us * 1e-6) / 1e9 if g_us else None
            out = {"workload": a.workload, "n": n, "nnz": nnz, "L": L, "hprec": p,
                   "apply_ms": t_apply * 1e3, "apply_GBs": tot / t_apply / 1e9,
                   "apply_frac": tot / t_apply / 1e9 / peak,
                   "gconv_us": g_us, "gconv_GBs": g_gbs,
                   "gconv_frac": g_gbs / peak if g_gbs else None,
                   "gconv_launches": info.gconv_launches, "layer_bytes": layer,
                   "peak_GBs": peak, "gen_s": gen_s, "l2_flushed": not a.warm,
                   "l2_bytes": torch.cuda.get_device_properties(0).L2_cache_size}
            print(json.dumps(out), flush=True)
        gnp.gnp_set_hprec(M, gnp.H_FP32)


if __name__ == "__main__":
    main()
