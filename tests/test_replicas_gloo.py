"""The N > 1 replica path on CPU: two gloo ranks, each with its own problem, no data-path
collective; the step time reported is the max over ranks and every rank's result is
the one it computes alone."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2406_00809_gb300 import inputs as I
    from paper_2406_00809_gb300 import replicas
    replicas.init("gloo")
    # each replica builds its own right-hand side; its "step time" differs per rank
    A = I.poisson2d(8)
    b = I.spmv(A, I.gaussian(A.n, seed=rank))
    local = float(np.linalg.norm(b))
    replicas.barrier()
    t = replicas.max_over_ranks(0.5 + rank)
    s = replicas.sum_over_ranks(1.0)
    out.put((rank, local, t, s))
    replicas.shutdown()


def test_two_gloo_replicas():
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
    for rank, local, t, s in res:
        assert t == 1.5 and s == 2.0
        assert local == pytest.approx(float(np.linalg.norm(I.spmv(A, I.gaussian(A.n, seed=rank)))), rel=0, abs=0)
