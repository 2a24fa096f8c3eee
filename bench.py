"""Benchmark: GNP-preconditioned FGMRES time-to-rtol on one GB300 (and replicas).

Workload (default): nonsymmetric 2-D convection-diffusion on a 256 x 256 grid
(n = 65,536, upwind, Peclet 100), GNP with hidden width 16 and 8 Res-GCONV layers in
float32, weights trained by this library (2,000 Adam steps, batch 16, half Eq. 5
Arnoldi samples with m = 40 and half N(0, I)), FGMRES(30) to rtol 1e-8 from x0 = 0,
b = A x with x ~ N(0, 1) (seed 0).  Synthetic inputs (no dataset).

One step = one complete solve.  Timed with CUDA events on the solve's stream after an
L2 flush (a 256 MB write); W untimed warm-up solves first.  Also reported:
* roofline of the dominant kernel (the Res-GCONV layer): CUDA events recorded around
  every Res-GCONV launch inside the captured restart cycle during a second pass of K
  solves (the event records slow the solve slightly, so the headline time comes from
  the first pass without them);
* e2e: the same solves with b copied from pinned host memory and x copied back inside
  the timed region;
* the bf16 hidden-block form of the same trained GNP (time-to-rtol, iterations);
* cpu_baseline: the float64 oracle on the host cores, a bounded sample of FGMRES
  iterations scaled to seconds per solve by this run's iteration count.
With --impl reference the oracle alone runs as the reference arm.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1: launched by torch.distributed.run, one replica solve per GPU (the path does not
shard: replicas only); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2406_00809_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    "convdiff256": dict(desc="2-D convection-diffusion 256x256 upwind Pe=100 (n=65,536)",
                        make=lambda: I.convdiff2d(256, 100.0), L=8, restart=30, rtol=1e-8,
                        maxiters=3000, train_steps=2000, batch=16, arnoldi_m=40),
    "powerlaw1m": dict(desc="power-law general sparse n=2^20 (mean 12, max 2000 nnz/row), row scaling 1e6",
                       make=lambda: I.powerlaw(1 << 20, seed=0), L=8, restart=50, rtol=1e-8,
                       maxiters=3000, train_steps=200, batch=16, arnoldi_m=40),
}
# iterations to rtol 1e-8 that the trained GNP of this library needs on each workload
# (measured by this bench's own arm: 651-672 on the convection-diffusion workload; the
# power-law one stops at the 3000-iteration cap); the reference arm scales its
# per-iteration time by it to report seconds per solve.
REF_ITERS = {"convdiff256": 660, "powerlaw1m": 3000}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def clocks_start(log_path=None):
    """Start sampling nvidia-smi clocks every 200 ms; the raw samples also go to log_path
    (CSV) when one is given."""
    try:
        f = open(log_path or os.devnull, "w")
    except OSError:
        f = open(os.devnull, "w")
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None, f
    return p, f


def clocks_stop(p, f, dev_index):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
        out, _ = p.communicate()
    f.write(out)
    f.close()
    sm, mx, reasons = [], None, set()
    for line in out.splitlines():
        parts = [t.strip() for t in line.split(",")]
        if len(parts) < 9 or parts[0] != str(dev_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def gconv_source_hash():
    """Hash of the sources that define the Res-GCONV kernel (a stored ncu traffic figure
    is used only while they are unchanged)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("gconv.cu", "common.cuh", "internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2406_00809_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def stored_traffic(workload):
    """DRAM bytes per Res-GCONV launch from the committed ncu summary, or None when the
    kernel sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", "res_gconv_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("source_hash") != gconv_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def gconv_kernel_name(A):
    """The Res-GCONV kernel the library picks for A: the short-row kernel when no row has
    more than 16 nonzeros (ROW_DMAX in csrc/gconv.cu), else the nnz-balanced tile kernel."""
    deg = int(np.max(np.diff(A.row_ptr))) if A.n else 0
    return ("k_gconv_row (Res-GCONV layer, short-row kernel)" if deg <= 16
            else "k_gconv (Res-GCONV layer, nnz-balanced tile kernel)")


def gconv_bytes(n, nnz, hbytes):
    """Algorithmic bytes of one Res-GCONV launch: row pointers, column indices and
    A_hat values (int32 + float32 per nonzero), the hidden block read once and the
    next one written once."""
    return 4 * (n + 1) + 8 * nnz + 2 * n * 16 * hbytes


# ----------------------------------------------------------------------- oracle arm

def oracle_sample(A, b, L, restart, seconds=15.0, maxit=60):
    """Time oracle FGMRES(restart) iterations with a Gaussian-init GNP (cost does not
    depend on the weight values) for about `seconds`; returns (seconds per iteration,
    iterations timed)."""
    from oracle import gnp_ref as G
    from oracle import krylov_ref as K
    Ah = G.normalise(A.to_scipy())
    P = G.unpack(I.init_weights(L, seed=0), L)
    As = A.to_scipy()
    it = 2
    total_t, total_it = 0.0, 0
    while total_t < seconds and it <= maxit:
        t0 = time.perf_counter()
        K.fgmres(As, b, lambda v: G.forward(Ah, v, P, 0), m=restart, rtol=1e-30, maxiters=it)
        dt = time.perf_counter() - t0
        total_t += dt
        total_it += it
        it *= 2
    return total_t / max(total_it, 1), total_it


def run_reference(args, wl):
    ws, rank, _ = dist_setup()
    if ws > 1 and rank != 0:
        return
    A = wl["make"]()
    x_true = I.gaussian(A.n, seed=0)
    b = I.spmv(A, x_true)
    iters = REF_ITERS[args.workload]
    per_step = []
    for s in range(args.warmup + args.steps):
        spi, nit = oracle_sample(A, b, wl["L"], wl["restart"], seconds=args.ref_seconds)
        if s >= args.warmup:
            per_step.append(spi * iters)
    value = statistics.mean(per_step)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "GNP-FGMRES time-to-rtol 1e-8 (s)", "value": value, "unit": "s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "L": wl["L"], "restart": wl["restart"], "rtol": wl["rtol"]},
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": f"float64 numpy/scipy oracle: FGMRES({wl['restart']}) + GNP iterations "
                                   f"timed for ~{args.ref_seconds:.0f} s per step, scaled by {iters} "
                                   "iterations to rtol (the iteration count of this library's trained GNP)"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------- our arm

def run_ours(args, wl):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_setup()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    A = wl["make"]()
    n, nnz = A.n, A.nnz
    x_true = I.gaussian(n, seed=0)
    b_np = I.spmv(A, x_true)
    L, m, rtol, maxit = wl["L"], wl["restart"], wl["rtol"], wl["maxiters"]
    with torch.cuda.stream(stream):
        Mt = gnp.mat_from_csr(A)
        cfg = gnp.make_config(L=L, batch=wl["batch"], arnoldi_m=wl["arnoldi_m"], seed=0)
        M = gnp.gnp_create(Mt, cfg, I.init_weights(L, seed=0))
        # construction: GNP training (outside the timed region, reported separately)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best = gnp.gnp_train(M, args.train_steps if args.train_steps is not None else wl["train_steps"])
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        b = torch.from_numpy(b_np).to(dev)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

        def solve(prof=False):
            x.zero_()
            return gnp.fgmres_solve(Mt, b, x, M, restart=m, rtol=rtol, maxiters=maxit, stream=stream,
                                    history=False)

        def timed_solves(k, prof=False):
            gnp.gnp_profile_gconv(prof)
            times, infos = [], []
            for _ in range(k):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                stream.synchronize()
                e0.record(stream)
                info = solve()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                infos.append(info)
            gnp.gnp_profile_gconv(False)
            return times, infos

        for _ in range(args.warmup):
            solve()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk, clkf = clocks_start(args.clocks_log) if rank == 0 else (None, None)
        times, infos = timed_solves(args.steps)
        clocks = clocks_stop(clk, clkf, local) if rank == 0 else None
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t_local = statistics.mean(times)
        if ws > 1:
            tt = torch.tensor([t_local], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_max = float(tt.item())
        else:
            t_max = t_local
        info = infos[-1]
        rel_true = float(np.linalg.norm(b_np - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b_np))
        # roofline pass: the same solves with the Res-GCONV launches event-timed
        rtimes, rinfos = timed_solves(max(1, args.steps), prof=True)
        g_ms = sum(i.gconv_ms for i in rinfos)
        g_n = sum(i.gconv_launches for i in rinfos)
        avg_launch_s = (g_ms / max(g_n, 1)) / 1e3
        # per-launch algorithmic bytes: L-1 plain layers + the decoder-fused last layer
        # (writes z, 4 bytes per row, instead of the next hidden block)
        per_solve_bytes = (L - 1) * gconv_bytes(n, nnz, 4) + (4 * (n + 1) + 8 * nnz + n * 16 * 4 + 4 * n)
        achieved = (per_solve_bytes / L) / avg_launch_s / 1e9 if g_n else None
        peak, peak_kind = load_peaks()
        # e2e: host buffers, copies inside the timed region
        b_host = torch.from_numpy(b_np).pin_memory()
        x_host = torch.empty(n, dtype=torch.float64).pin_memory()
        e2e_times = []
        for _ in range(args.steps):
            flush.zero_()
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.copy_(b_host, non_blocking=True)
            x.zero_()
            gnp.fgmres_solve(Mt, b, x, M, restart=m, rtol=rtol, maxiters=maxit, stream=stream, history=False)
            x_host.copy_(x, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e2e_times.append(e0.elapsed_time(e1) / 1e3)
        # bf16 hidden block form of the same trained GNP
        gnp.gnp_set_hprec(M, gnp.H_BF16)
        for _ in range(max(1, args.warmup)):
            solve()
        btimes, binfos = timed_solves(args.steps)
        gnp.gnp_set_hprec(M, gnp.H_FP32)
    # kernel launches inside the timed region: per cycle m steps of (encode, which from
    # step 1 on also forms the basis vector and finishes the previous step; L Res-GCONV
    # with the decoder in the last; SpMV + CGS2 pass 1; pass 2) + the last step's finish
    # + x update + residual; per solve + norm and initial residual
    per_cycle = m * (L + 3) + 3
    launches = sum(i.cycles * per_cycle + 2 for i in infos)
    line = {
        "metric": "GNP-FGMRES time-to-rtol 1e-8 (s)", "value": t_max, "unit": "s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n": n, "nnz": nnz, "L": L, "hidden": 16, "hprec": "fp32",
                   "restart": m, "rtol": rtol, "train_steps": args.train_steps or wl["train_steps"],
                   "batch": wl["batch"], "arnoldi_m": wl["arnoldi_m"], "x0": "zeros",
                   "l2": "flushed (256 MB write) before every timed solve", "parallelism": f"replicas{ws}"},
        "iters": info.iters, "status": info.status_name, "rel_res_true": rel_true,
        "solves_per_s": ws / t_max,
        "train": {"steps": args.train_steps or wl["train_steps"], "seconds": train_s, "best_loss": best},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": stored_traffic(args.workload),
                     "kernel": gconv_kernel_name(A), "peak_kind": peak_kind,
                     "bytes_per_launch": per_solve_bytes / L, "launches_timed": g_n,
                     "avg_launch_us": avg_launch_s * 1e6},
        "e2e": {"value": statistics.mean(e2e_times), "unit": "s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "bf16": {"value": statistics.mean(btimes), "unit": "s", "iters": binfos[-1].iters,
                 "status": binfos[-1].status_name},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        spi, nit = oracle_sample(A, b_np, L, m, seconds=args.ref_seconds)
        line["cpu_baseline"] = {"value": spi * info.iters, "unit": "s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"{nit} float64 oracle FGMRES({m})+GNP iterations (numpy/scipy, "
                                          f"default threading), {spi*1e3:.1f} ms each, scaled by this run's "
                                          f"{info.iters} iterations"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="convdiff256")
    ap.add_argument("--train-steps", type=int, default=None)
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-log", default=None, help="also write the raw clock samples (CSV) here")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
