"""Serving benchmark: p50/p99 latency and solves/s of the continuous-batching server.

    python -m paper_2406_00809_gb300.serve_bench [--requests 128] [--load 0.25,0.5,1,2]
        [--pool 12] [--nmin 1e4] [--nmax 2e6] [--train-steps 300] [--hprec bf16]

A pool of `pool` problems is built first (not timed): the three generator families
(2-D Poisson, 2-D convection-diffusion, power-law general sparse, the latter with the
diagonal shift --powerlaw-shift times its spectral radius when given) in turn, n drawn
log-uniformly in [nmin, nmax] (grid side round(sqrt(n)) for the 2-D families), each
with its own GNP (8 layers, hidden 16) trained for `train_steps` Adam steps on its own
matrix and then applied with a bfloat16 hidden block.  Each of the `requests` solves
picks a pool problem uniformly and has its own right-hand side b = A x, x ~ N(0, 1)
(device generator seeded by the request index); FGMRES(30) to rtol 1e-8, at most
`maxiters` steps.  Requests arrive as a Poisson process at each swept rate (solves per
second); latency = submit to finish, measured by the server's steady clock.  A pool
(not a fresh matrix per request) keeps the set-up time bounded; every request still
runs with its own workspace, right-hand side and solution.

The arrival rates are multiples (--load) of the sequential capacity: one solve of every
pool problem is first run alone through the server, and 1 / (mean solo latency) is the
rate at which requests served one at a time would just keep up.  Load 1 and above
therefore measure how much concurrent requests gain over serial service.  One JSON line
per rate (plus one with the solo latencies).  --grouped 1 runs the server in grouped mode
(the Poisson and convection-diffusion requests advance in grouped steps, the power-law
ones, whose long rows need the tile kernels, per request).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_00809_gb300 import inputs as I  # noqa: E402


def build_pool(g, args, rng):
    import torch
    pool = []
    fams = ["poisson", "convdiff", "powerlaw"]
    for i in range(args.pool):
        fam = fams[i % 3]
        n = float(np.exp(rng.uniform(np.log(args.nmin), np.log(args.nmax))))
        if fam == "poisson":
            A = I.poisson2d(max(8, int(round(np.sqrt(n)))))
        elif fam == "convdiff":
            A = I.convdiff2d(max(8, int(round(np.sqrt(n)))), 100.0)
        else:
            A = I.powerlaw(max(64, int(n)), seed=100 + i, shift_fraction=getattr(args, "powerlaw_shift", None))
        Mt = g.mat_from_csr(A)
        M = g.gnp_create(Mt, g.make_config(L=8, batch=args.batch, arnoldi_m=20, seed=i),
                         I.init_weights(8, seed=i))
        t0 = time.perf_counter()
        if args.train_steps > 0:
            g.gnp_train(M, args.train_steps)
        g.gnp_train_release(M)
        g.gnp_set_hprec(M, g.H_BF16 if args.hprec == "bf16" else g.H_FP32)
        torch.cuda.synchronize()
        pool.append(dict(fam=fam, n=A.n, nnz=A.nnz, A=Mt, M=M, train_s=time.perf_counter() - t0))
    return pool


def run_rate(g, srv, pool, args, rate, seed):
    import torch
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(pool), size=args.requests)
    gaps = rng.exponential(1.0 / rate, size=args.requests)
    arrivals = np.cumsum(gaps)
    bufs = []
    for r, k in enumerate(picks):
        p = pool[k]
        gen = torch.Generator(device="cuda").manual_seed(int(seed * 100000 + r))
        xt = torch.randn(p["n"], dtype=torch.float64, device="cuda", generator=gen)
        b = torch.empty_like(xt)
        g.gnp_spmv(p["A"], xt, b)
        bufs.append((b, torch.zeros_like(xt)))
    torch.cuda.synchronize()
    tickets = [None] * args.requests
    t_start = time.perf_counter()

    def submitter():
        for r, k in enumerate(picks):
            delay = t_start + arrivals[r] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            p = pool[k]
            tickets[r] = srv.submit(p["A"], p["M"], bufs[r][0], bufs[r][1], args.rtol, args.maxiters)

    th = threading.Thread(target=submitter)
    th.start()
    results = [None] * args.requests
    done = 0
    while done < args.requests:
        progressed = False
        for r in range(args.requests):
            if results[r] is None and tickets[r] is not None:
                res = srv.poll(tickets[r])
                if res is not None:
                    results[r] = res
                    done += 1
                    progressed = True
        if not progressed:
            time.sleep(0.0005)
    th.join()
    t_end = time.perf_counter()
    lat = np.array([res.seconds for res in results])
    its = np.array([res.iters for res in results])
    status = {}
    by_family = {}
    for k, res in zip(picks, results):
        status[res.status_name] = status.get(res.status_name, 0) + 1
        fam = by_family.setdefault(pool[k]["fam"], {})
        fam[res.status_name] = fam.get(res.status_name, 0) + 1
    ok = np.array([res.status_name == "GNP_OK" for res in results])
    st = srv.stats()
    return {"rate_per_s": rate, "requests": args.requests, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "solves_per_s": args.requests / (t_end - t_start), "iters_mean": float(its.mean()),
            "iters_max": int(its.max()), "status": status, "status_by_family": by_family,
            "p50_s_converged": float(np.percentile(lat[ok], 50)) if ok.any() else None,
            "p99_s_converged": float(np.percentile(lat[ok], 99)) if ok.any() else None,
            "max_active_seen": st["max_active_seen"], "rounds": st["rounds"]}


def solo_latencies(g, srv, pool, args):
    """Each pool problem solved alone through the server (after a warm-up solve that
    captures its graphs): its latency, iterations and status."""
    import torch
    out = []
    for k, p in enumerate(pool):
        gen = torch.Generator(device="cuda").manual_seed(10_000 + k)
        xt = torch.randn(p["n"], dtype=torch.float64, device="cuda", generator=gen)
        b = torch.empty_like(xt)
        g.gnp_spmv(p["A"], xt, b)
        x = torch.zeros_like(xt)
        srv.wait(srv.submit(p["A"], p["M"], b, x, args.rtol, args.maxiters))
        x.zero_()
        res = srv.wait(srv.submit(p["A"], p["M"], b, x, args.rtol, args.maxiters))
        out.append(dict(n=p["n"], fam=p["fam"], seconds=res.seconds, iters=res.iters, status=res.status_name))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=128)
    ap.add_argument("--load", default="0.25,0.5,1,2",
                    help="arrival rates as multiples of the sequential capacity")
    ap.add_argument("--pool", type=int, default=12)
    ap.add_argument("--nmin", type=float, default=1e4)
    ap.add_argument("--nmax", type=float, default=2e6)
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--hprec", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--maxiters", type=int, default=1000)
    ap.add_argument("--powerlaw-shift", type=float, default=None,
                    help="diagonal shift of the power-law family as a fraction of its spectral radius "
                         "(default: the calibrated cond ~1e6 shift)")
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--max-gb", type=float, default=120.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--rates", default=None,
                    help="absolute arrival rates (solves/s), in place of --load (to compare server modes)")
    ap.add_argument("--grouped", type=int, default=0, choices=[0, 1],
                    help="1: grouped steps for the requests whose GNP runs on the short-row kernels")
    a = ap.parse_args()
    import torch
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp as g
    rng = np.random.default_rng(a.seed)
    t0 = time.perf_counter()
    pool = build_pool(g, a, rng)
    setup_s = time.perf_counter() - t0
    print(json.dumps({"pool": [{k: p[k] for k in ("fam", "n", "nnz", "train_s")} for p in pool],
                      "setup_s": setup_s}), flush=True)
    srv = g.Server(max_bytes=int(a.max_gb * (1 << 30)), max_active=a.max_active, restart=30,
                   grouped=bool(a.grouped))
    solo = solo_latencies(g, srv, pool, a)
    capacity = 1.0 / float(np.mean([s_["seconds"] for s_ in solo]))
    print(json.dumps({"solo": solo, "sequential_capacity_per_s": capacity}), flush=True)
    rates = ([float(r) for r in a.rates.split(",")] if a.rates
             else [float(r) * capacity for r in a.load.split(",")])
    for i, rate in enumerate(rates):
        load = rate / capacity
        out = run_rate(g, srv, pool, a, rate, a.seed + 1 + i)
        out.update({"metric": "serve latency", "load": load, "hprec": a.hprec, "pool": a.pool, "grouped": a.grouped,
                    "n_range": [a.nmin, a.nmax], "train_steps": a.train_steps})
        print(json.dumps(out), flush=True)
    srv.close()


if __name__ == "__main__":
    main()
