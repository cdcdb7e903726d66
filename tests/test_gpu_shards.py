"""The product's sampling pass sharded across ranks (GPU).

A pass over [start, start + n) equals the sum of passes over any split of
that range (the paper's n/N points per core, Sect. 2.1): two gloo ranks each
run cv_sample on their own contiguous share (independent launches on the one
GPU, nothing waits on another rank's kernel), one all-reduce of S1, S2 and
the histogram on the host gives the pass, and that equals the library's
single pass and the FP64 oracle's.  Exact for f = 1 on the uniform grid
(the counts), to the order of additions otherwise."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NDIM, N, START, NPTS = 5, 64, 12345, 300001


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(cg, family):
    rng = np.random.default_rng(21)
    a = 0.5 + rng.random((2, NDIM))
    u = rng.random((2, NDIM))
    if family == "const":
        return cg.genz(NDIM, [cg.CONST, cg.CONST], a, u), a, u
    return cg.genz(NDIM, [cg.GAUSSIAN, cg.C0], a, u), a, u


def _edges(family):
    e = np.tile(np.linspace(0.0, 1.0, N + 1), (NDIM, 1))
    if family != "const":
        e[:, 1:-1] += 0.003 * np.sin(np.arange(1, N))[None, :]  # a non-uniform grid
    return e


def _pass(cg, ctx, g, family, lo, cnt, flags):
    e = torch.tensor(_edges(family), dtype=torch.float64, device="cuda")
    S1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((NDIM, N), dtype=torch.float64, device="cuda")
    ctx.sample(g, N, e, lo, cnt, flags, S1, S2, H)
    ctx.synchronize()
    return torch.cat([S1, S2, H.ravel()]).cpu()


def _worker(rank, world, port, family, flags, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1408_6373_gb300 as cg
    cg.build_library()
    ctx = cg.Context(0)
    g, _, _ = _problem(cg, family)
    share = NPTS // world
    lo = START + rank * share
    cnt = share if rank < world - 1 else NPTS - (world - 1) * share
    t = _pass(cg, ctx, g, family, lo, cnt, flags)
    dist.all_reduce(t)
    if rank == 0:
        out.put((t.numpy().copy(), _pass(cg, ctx, g, family, START, NPTS, flags).numpy()))
    dist.barrier()
    ctx.close()
    dist.destroy_process_group()


def _run(family, flags):
    mpc = mp.get_context("spawn")
    q = mpc.SimpleQueue()
    port = _free_port()
    procs = [mpc.Process(target=_worker, args=(r, 2, port, family, flags, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got, full = q.get()
    for pr in procs:
        pr.join(300)
        assert pr.exitcode == 0
    return got, full


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("flags", [0, 0x100], ids=["fp32", "fp64"])
def test_constant_integrand_shards_count_exactly(gpu, flags):
    got, full = _run("const", flags)
    # f = 1 on the uniform grid of 2^6 bins: J = 1 exactly, so S1 = S2 = the
    # number of points and H the number of points in each bin, in any split
    np.testing.assert_array_equal(got, full)
    assert got[0] == NPTS and got[2] == NPTS
    H = got[4:].reshape(NDIM, N)
    assert np.all(H.sum(axis=1) == NPTS) and np.all(H == np.round(H))


@pytest.mark.parametrize("flags", [0x100], ids=["fp64"])
def test_two_rank_product_shards_match_full_pass_and_oracle(gpu, flags):
    import oracle as O
    import paper_1408_6373_gb300 as cg
    got, full = _run("genz", flags)
    np.testing.assert_allclose(got, full, rtol=1e-12, atol=1e-300)
    _, a, u = _problem(cg, "genz")
    p = O.Problem(NDIM, [O.GAUSSIAN, O.C0], a, u, nbins=N)
    S1, S2, H = O.sample(p, _edges("genz"), START, NPTS)
    ref = np.concatenate([S1, S2, H.ravel()])
    np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12)
    hmax = np.abs(ref[4:]).reshape(NDIM, N).max(axis=1, keepdims=True)
    assert np.all(np.abs(got[4:] - ref[4:]).reshape(NDIM, N) <= 1e-12 * hmax)
