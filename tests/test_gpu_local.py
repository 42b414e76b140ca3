"""GPU parity of local alignment (nw_local_align_batch, Smith-Waterman)
against the CPU oracle: scores, start and end cells and CIGARs bit-exact,
over ragged lengths, every rows-per-lane shape, several scorings, pointer
waves under a small budget, device buffers, and the 4,000-pair local
workload of the benchmark."""
import os

import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu

LENGTHS = [0, 1, 2, 31, 32, 33, 95, 96, 97, 255, 256, 257, 300, 513, 1000, 1500]


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream())
    yield c
    c.close()


def _pool(pairs):
    import paper_2412_21103_gb300 as nw
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    return pool, off[0::2], lens[0::2], off[1::2], lens[1::2]


def _pairs(seed, count):
    rs = seqgen.Stream(seed)
    out = []
    for k in range(count):
        m = LENGTHS[int(rs.integers(0, len(LENGTHS) - 1, 1)[0])]
        n = LENGTHS[int(rs.integers(0, len(LENGTHS) - 1, 1)[0])]
        if k % 3 == 0 and m > 8:
            p = seqgen.long_mutated_pair(seed * 100 + k, m=m)
            lo = int(rs.integers(0, m // 4, 1)[0])
            out.append((p.a, p.b[lo: lo + max(n, 1)]))      # a shifted piece: a real local match
        else:
            out.append((rs.bases(m), rs.bases(n)))
    return out


def _check(got, want, with_cigar=True):
    scores, ends, cigars = got
    for k, (s, e, ops) in enumerate(want):
        assert int(scores[k]) == s, k
        assert tuple(int(x) for x in ends[k]) == e, k
        if with_cigar:
            assert cigars[k] == oracle.rle(ops), k


@pytest.mark.parametrize("rows", ["4", "8", "16"])
@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -3, -2), (1, -40, -40)])
def test_local_cigars_every_shape(ctx, rows, sc, monkeypatch):
    import paper_2412_21103_gb300 as nw
    monkeypatch.setenv("NW_LOCAL_R", rows)
    pairs = _pairs(40 + int(rows) + sc[1], 70)
    pool, ao, al, bo, bl = _pool(pairs)
    got = nw.nw_local_align_batch(ctx, pool, ao, al, bo, bl, sc, nw.NW_CIGAR)
    _check(got, oracle.local_align_many(pairs, *sc))


@pytest.mark.parametrize("rows", ["4", "8", "16"])
def test_local_scores_and_end_cells(ctx, rows, monkeypatch):
    """Score only: without ends, and with ends (the end cell; the start is
    not computed)."""
    import paper_2412_21103_gb300 as nw
    monkeypatch.setenv("NW_LOCAL_R", rows)
    pairs = _pairs(90 + int(rows), 90)
    pool, ao, al, bo, bl = _pool(pairs)
    scores, ends, _ = nw.nw_local_align_batch(ctx, pool, ao, al, bo, bl, (1, -1, -1), 0)
    want = oracle.local_align_many(pairs)
    for k, (s, e, _) in enumerate(want):
        assert int(scores[k]) == s, k
        assert tuple(int(x) for x in ends[k][2:]) == e[2:], k
        assert tuple(int(x) for x in ends[k][:2]) == (0xFFFFFFFF, 0xFFFFFFFF)


def test_local_waves_under_a_small_budget():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream(), mem_budget=48 << 20)
    pairs = [(p.a, p.b) for p in seqgen.local_pairs(77, 12, ref_min=3000, ref_max=6000, win_min=1000, win_max=3000)]
    pool, ao, al, bo, bl = _pool(pairs)
    got = nw.nw_local_align_batch(c, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR)
    _check(got, oracle.local_align_many(pairs))
    c.close()


def test_local_device_buffers(ctx):
    import torch
    import paper_2412_21103_gb300 as nw
    pairs = [(p.a, p.b) for p in seqgen.local_pairs(78, 40, ref_min=500, ref_max=3000, win_min=100, win_max=800)]
    pool, ao, al, bo, bl = _pool(pairs)
    n = len(pairs)
    coff = nw._cigar_offsets(al, bl)
    scores = torch.zeros(n, dtype=torch.int32, device="cuda")
    ends = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    cpool = torch.zeros(int(coff[-1]), dtype=torch.uint8, device="cuda")
    clen = torch.zeros(n, dtype=torch.int64, device="cuda")
    nw.nw_local_align_batch(ctx, torch.from_numpy(pool).cuda(), ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR, scores,
                            ends, cpool, coff, clen)
    ctx.sync()
    cp, cl = cpool.cpu().numpy(), clen.cpu().numpy()
    got = (scores.cpu().numpy(), ends.cpu().numpy().astype(np.uint32),
           [cp[int(coff[k]): int(coff[k]) + int(cl[k])].tobytes().decode() for k in range(n)])
    _check(got, oracle.local_align_many(pairs))


def test_local_workload_full_size(ctx):
    """The benchmark's workload: 4,000 pairs of a mutated reference window
    between random flanks against its 2-10 kb reference (seed 1006).  Every
    score against the oracle; start, end and CIGAR of 200 pairs (the
    longest, the widest and random) against the oracle."""
    import paper_2412_21103_gb300 as nw
    pairs = [(p.a, p.b) for p in seqgen.local_pairs(1006, 4000)]
    pool, ao, al, bo, bl = _pool(pairs)
    scores, ends, cigars = nw.nw_local_align_batch(ctx, pool, ao, al, bo, bl, (1, -1, -1), nw.NW_CIGAR)
    assert scores.tolist() == oracle.local_score_many(pairs)
    cells = al.astype(np.int64) * bl.astype(np.int64)
    rs = seqgen.Stream(5150)
    sample = sorted(set(np.argsort(-cells)[:40].tolist()) | set(np.argsort(-al.astype(np.int64))[:40].tolist()) |
                    set(int(k) for k in rs.integers(0, len(pairs) - 1, 120)))
    want = oracle.local_align_many([pairs[k] for k in sample])
    for k, (s, e, ops) in zip(sample, want):
        assert int(scores[k]) == s and tuple(int(x) for x in ends[k]) == e and cigars[k] == oracle.rle(ops), k
