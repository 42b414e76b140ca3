"""Pair sharding over ranks (the paper's Sec. 3.2 MPI split and gather):
the library's LPT partition on the host, and the all-gather of scores and
CIGAR bytes on two gloo ranks on the CPU, where each rank aligns its share
with the oracle in place of the GPU library (the GPU version of the same
run is in test_gpu_shard.py)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shard():
    from paper_2412_21103_gb300 import build
    build.build()
    from paper_2412_21103_gb300 import shard as sh
    return sh


def test_lpt_by_hand(shard):
    """Cells 10, 7, 6, 5, 4 on two ranks: 10 -> r0; 7 -> r1; 6 -> r1 (7 < 10,
    load 13); 5 -> r0 (10 < 13, load 15); 4 -> r1 (13 < 15, load 17)."""
    rank_of, loads = shard.shard_pairs([10, 7, 6, 5, 4], [1, 1, 1, 1, 1], 2)
    assert rank_of.tolist() == [0, 1, 1, 0, 1] and loads.tolist() == [15, 17]


def test_lpt_ties_go_to_the_lowest_rank_and_index(shard):
    rank_of, loads = shard.shard_pairs([5, 5, 5, 5, 0], [1, 1, 1, 1, 9], 3)
    assert rank_of.tolist() == [0, 1, 2, 0, 1] and loads.tolist() == [10, 5, 5]


@pytest.mark.parametrize("nranks", [1, 2, 3, 8])
def test_lpt_properties(shard, nranks):
    import seqgen
    rs = seqgen.Stream(50 + nranks)
    a = rs.integers(0, 3000, 500)
    b = rs.integers(0, 3000, 500)
    rank_of, loads = shard.shard_pairs(a, b, nranks)
    cells = a.astype(np.int64) * b.astype(np.int64)
    assert rank_of.max() < nranks
    per = np.bincount(rank_of, weights=cells, minlength=nranks)
    assert per.tolist() == loads.astype(np.float64).tolist()
    assert loads.sum() == cells.sum()
    assert loads.max() <= cells.sum() / nranks + cells.max()      # list scheduling bound


def test_rejects_zero_ranks(shard):
    import paper_2412_21103_gb300 as nw
    with pytest.raises(nw.NWError):
        shard.shard_pairs([1], [1], 0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pairs():
    sys.path.insert(0, ROOT)
    import seqgen
    rs = seqgen.Stream(808)
    out = []
    for k in range(37):
        m, n = int(rs.integers(0, 400, 1)[0]), int(rs.integers(0, 400, 1)[0])
        out.append((rs.bases(m), rs.bases(n)))
    return out


def _rank(rank, world, port, want_cigar, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    from paper_2412_21103_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pairs = _pairs()
        a_len = [p[0].size for p in pairs]
        b_len = [p[1].size for p in pairs]
        seen = []

        def aligner(idx):   # the oracle stands in for the GPU library on a CPU rank
            seen.extend(int(k) for k in idx)
            res = oracle.align_many([pairs[k] for k in idx])
            return [s for s, _ in res], ([oracle.rle(o) for _, o in res] if want_cigar else None)
        flags = 1 if want_cigar else 0
        scores, cigars, mine = sh.align_batch_sharded(None, None, np.zeros(len(pairs)), a_len, np.zeros(len(pairs)),
                                                      b_len, (1, -1, -1), flags, aligner=aligner)
        q.put((rank, scores.tolist(), cigars, sorted(seen), mine.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("want_cigar", [True, False])
def test_two_gloo_ranks_gather_every_result(want_cigar):
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, want_cigar, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    pairs = _pairs()
    want = oracle.align_many(pairs)
    shares = [g[3] for g in got]
    assert sorted(shares[0] + shares[1]) == list(range(len(pairs)))   # each pair on exactly one rank
    assert shares[0] and shares[1]
    for rank, scores, cigars, seen, mine in got:
        assert seen == mine
        assert scores == [s for s, _ in want]
        if want_cigar:
            assert cigars == [oracle.rle(o) for _, o in want]
        else:
            assert cigars is None
