"""The multi-rank path of bench.py on CPU: two gloo ranks, each decoding its own codeword range
with the oracle (standing in for the GPU decode), then the cross-rank operations the benchmark
uses: the barrier, the max of the step time and the sum of the statistics.  The sums must equal
one process decoding the union of the ranges."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")

N, K, BATCH, EBN0, MAX_ITER = 64, 32, 24, 2.0, 30


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _decode_range(first, count):
    from oracle import oracle as O
    from paper_1505_04979_gb300 import inputs as I
    fz = O.bec_frozen(N, K)
    idx = np.arange(first, first + count)
    u = I.info_bits(I.DEFAULT_SEED, idx, fz)
    llr = I.channel_llr(O.encode(u), I.gaussian(I.DEFAULT_SEED, idx, N), I.sigma(EBN0, K / N))
    uh, it, pe, _ = O.decode_batch(fz, llr, MAX_ITER, 0.9375, O.STOP_GMATRIX, O.FREEZE_CSFG, nthreads=1)
    errs = int((uh != u).any(axis=1).sum())
    return [errs, int((uh != u).sum()), float(it.sum()), float(pe.sum())]


def _rank(rank, world, port, out):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    r, local, w = bench.dist_setup(world)
    assert (r, local, w) == (rank, rank, world) and dist.get_backend() == "gloo"
    first = bench.shard_first(r, BATCH)
    stats = _decode_range(first, BATCH)
    bench.barrier(w)
    t = bench.max_over_ranks(0.25 + r, w)
    sums = bench.sum_over_ranks(stats, w)
    out.put((r, first, stats, sums, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, first, stats, sums, t = out.get(timeout=240)
        got[r] = (first, stats, sums, t)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][0] == 0 and got[1][0] == BATCH                      # disjoint, adjacent ranges
    assert got[0][3] == got[1][3] == 1.25                             # max of the ranks' times
    assert got[0][2] == got[1][2]                                     # every rank gets the sums
    assert got[0][2] == [a + b for a, b in zip(got[0][1], got[1][1])]
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    assert got[0][2] == _decode_range(0, 2 * BATCH)                   # = one process over the union
