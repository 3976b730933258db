"""Multi-process paths on CPU (gloo, world size 2).

* The bench's max-over-ranks timing reduction.
* The frequency-sharded MDC (the paper's partitioning of the kernel along frequency):
  each rank holds a slab of frequencies, computes its partial inverse transform, and one
  all-reduce (sum) of y completes the pass because the inverse FFT is linear.  The ranks
  use the FP64 oracle, so this checks the decomposition, not a kernel.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import mdc as omdc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def shard_forward(G, x, dt, dr, ks):
    """Partial forward MDC from the frequency bins ks only (zero elsewhere)."""
    nt = x.shape[0]
    X = omdc.rfft_truncate(x, G.shape[0])
    Y = np.zeros((G.shape[0], G.shape[1], x.shape[2]), complex)
    Y[ks] = np.matmul(G[ks] * (dt * dr), X[ks])
    return omdc.pad_irfft(Y, nt)


def test_frequency_shards_sum_to_full_operator():
    rng = np.random.default_rng(0)
    nt, nf, nr, ns, nv = 64, 20, 6, 7, 2
    G = rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))
    x = rng.standard_normal((nt, ns, nv))
    full = omdc.forward(G, x, 0.004, 400.0)
    parts = [shard_forward(G, x, 0.004, 400.0, ks) for ks in np.array_split(np.arange(nf), 3)]
    assert np.linalg.norm(sum(parts) - full) <= 1e-13 * np.linalg.norm(full)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    try:
        # timing reduction used by bench.py under torchrun
        got = bench.max_over_ranks([1.0 + rank, 5.0 - rank], "cpu")
        # frequency-sharded forward with one all-reduce
        rng = np.random.default_rng(1)
        nt, nf, nr, ns, nv = 64, 17, 5, 8, 3
        G = rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))
        x = rng.standard_normal((nt, ns, nv))
        import paper_2011_11120_gb300 as m
        k0, nk = m.shard_bounds(nf, world, rank)        # the library's band split (host logic)
        ks = np.arange(k0, k0 + nk)
        y = torch.from_numpy(shard_forward(G, x, 0.004, 400.0, ks))
        dist.all_reduce(y, op=dist.ReduceOp.SUM)
        full = omdc.forward(G, x, 0.004, 400.0)
        err = float(np.linalg.norm(y.numpy() - full) / np.linalg.norm(full))
        q.put((rank, got, err))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=100) for _ in procs]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, got, err in res:
        assert got == [2.0, 5.0]
        assert err <= 1e-13


def test_shard_bounds_tile_the_band():
    """The band split gives contiguous, disjoint bands covering 0 .. nf-1, sizes differing by
    at most one, and rejects more ranks than bins."""
    import paper_2011_11120_gb300 as m
    for nf in (1, 2, 7, 150, 300, 513):
        for world in range(1, min(nf, 9) + 1):
            b = [m.shard_bounds(nf, world, r) for r in range(world)]
            assert b[0][0] == 0 and sum(nk for _, nk in b) == nf
            assert all(b[i][0] + b[i][1] == b[i + 1][0] for i in range(world - 1))
            assert max(nk for _, nk in b) - min(nk for _, nk in b) <= 1
    with pytest.raises(ValueError):
        m.shard_bounds(3, 4, 0)
