"""Multi-process paths on the CPU (gloo, world size 2).

The sampling pass shards: every rank samples its own contiguous part of an
iteration's Sobol index range (the paper's "n/N points per core",
Sect. 2.1), and one all-reduce of S1, S2 and the histogram gives the
iteration.  This checks that invariance with the oracle on two ranks, and
the benchmark's max-over-ranks reduction of the step time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    import bench
    ndim, N, start, n = 4, 32, 7, 20001
    p = O.Problem(ndim, [O.GAUSSIAN, O.C0], np.full((2, ndim), 2.0), np.full((2, ndim), 0.4), nbins=N)
    e = O.grid_uniform(ndim, N)
    e[:, 1:-1] += 0.01 * np.sin(np.arange(1, N))  # a non-uniform grid
    lo = start + rank * (n // world)
    cnt = n // world if rank < world - 1 else n - (world - 1) * (n // world)
    S1, S2, H = O.sample(p, e, lo, cnt)
    t = torch.tensor(np.concatenate([S1, S2, H.ravel()]), dtype=torch.float64)
    dist.all_reduce(t)
    mx = bench.max_over_ranks(float(rank + 1))
    if rank == 0:
        full = np.concatenate([*O.sample(p, e, start, n)[:2], O.sample(p, e, start, n)[2].ravel()])
        out.put((t.numpy().copy(), full, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_sum_to_the_full_pass():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got, full, mx = q.get()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    np.testing.assert_allclose(got, full, rtol=1e-13, atol=1e-300)
    assert mx == 2.0
