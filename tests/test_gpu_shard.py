"""Pair sharding with the GPU library (the paper's Sec. 3.2 split and
gather): two ranks, each a process with its own context on the one GPU of
this box, align their LPT shares with nw_align_batch and all-gather the
scores and CIGAR bytes over gloo (host tensors: the collective never reads
GPU memory).  The two ranks' kernels do not wait on each other, so they may
share a GPU.  Every gathered result equals the oracle's, and equals one
unsharded batch."""
import os
import socket
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pairs():
    sys.path.insert(0, ROOT)
    import seqgen
    return [(p.a, p.b) for p in seqgen.band_pairs(1004, npairs=60, lmin=300, lmax=4000)]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_2412_21103_gb300 as nw
    from paper_2412_21103_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ctx = nw.Context(0, torch.cuda.current_stream())
        seqs = []
        for a, b in _pairs():
            seqs += [a, b]
        pool, off, lens = nw.pool_of(seqs)
        scores, cigars, mine = sh.align_batch_sharded(ctx, pool, off[0::2], lens[0::2], off[1::2], lens[1::2],
                                                      (1, -1, -1), nw.NW_CIGAR | nw.NW_LEARNED_BAND)
        ctx.close()
        q.put((rank, scores.tolist(), cigars, mine.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_the_pairs_and_gather_exact_results():
    import torch.multiprocessing as mp
    import oracle
    import paper_2412_21103_gb300 as nw
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=300) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=120)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    pairs = _pairs()
    want = oracle.align_many(pairs)
    assert sorted(got[0][3] + got[1][3]) == list(range(len(pairs)))
    for _, scores, cigars, _ in got:
        assert scores == [s for s, _ in want]
        assert cigars == [oracle.rle(o) for _, o in want]
    # and one unsharded call of this process
    import torch
    c = nw.Context(0, torch.cuda.current_stream())
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    s1, c1 = nw.nw_align_batch(c, pool, off[0::2], lens[0::2], off[1::2], lens[1::2], (1, -1, -1), nw.NW_CIGAR)
    c.close()
    assert s1.tolist() == got[0][1] and c1 == got[0][2]
