"""The N > 1 replica path of bench.py on CPU: two gloo ranks, each with its own problem,
no data-path collective.  bench.aggregate (through paper_2406_00809_gb300.replicas, the
code bench.py runs under torch.distributed.run) must report the max over ranks of the
step time and the sum over ranks of the solves, and every rank's result is the one it
computes alone."""
import importlib.util
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2406_00809_gb300 import inputs as I
    from paper_2406_00809_gb300 import replicas
    bench = _load_bench()
    assert replicas.env() == (world, rank, rank)
    assert replicas.init("gloo") == world
    # each replica builds its own right-hand side; its "step time" differs per rank
    A = I.poisson2d(8)
    b = I.spmv(A, I.gaussian(A.n, seed=rank))
    local = float(np.linalg.norm(b))
    replicas.barrier()
    t, solves = bench.aggregate(0.5 + rank, 1.0 + rank)
    out.put((rank, local, t, solves))
    replicas.shutdown()


def test_two_gloo_replicas_through_bench_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2406_00809_gb300 import inputs as I
    A = I.poisson2d(8)
    for rank, local, t, solves in res:
        assert t == 1.5 and solves == 3.0
        assert local == pytest.approx(float(np.linalg.norm(I.spmv(A, I.gaussian(A.n, seed=rank)))), rel=0, abs=0)


def test_single_process_aggregate_is_identity():
    bench = _load_bench()
    assert bench.aggregate(0.25, 4.0) == (0.25, 4.0)
