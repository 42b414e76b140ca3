"""Autotuner and CUDA-graph replay (a7): tuned shapes and replayed graphs
give the oracle's results, the tuning table records one choice per workload
signature and can be preloaded, and a replayed graph re-reads the sequence
pool (new contents, same buffers: new, exact scores)."""
import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu


def _family(seed, nseq, lmin=60, lmax=400):
    rs = seqgen.Stream(seed)
    return [rs.bases(int(L)) for L in rs.integers(lmin, lmax, nseq)]


def _matrix_oracle(seqs, sc=(1, -1, -1)):
    n = len(seqs)
    pairs = [(seqs[i], seqs[j]) for i in range(n) for j in range(i + 1, n)]
    got = oracle.score_many(pairs, *sc)
    M = np.zeros((n, n), np.int32)
    k = 0
    for i in range(n):
        M[i, i] = seqs[i].size * sc[0]
        for j in range(i + 1, n):
            M[i, j] = M[j, i] = got[k]
            k += 1
    return M


def test_autotuned_all_pairs_exact_and_recorded():
    import torch
    import paper_2412_21103_gb300 as nw
    seqs = _family(71, 40)
    pool, off, lens = nw.pool_of(seqs)
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        ctx.set_autotune(True)
        M1 = nw.nw_score_all_pairs(ctx, pool, off, lens)
        table = ctx.tuning()
        M2 = nw.nw_score_all_pairs(ctx, pool, off, lens)
        assert ctx.tuning() == table  # the second call reuses the choice
    keys = [k for k in table if k.startswith("batch_rows:")]
    assert len(keys) == 1 and table[keys[0]] in (4, 8, 16, 32)  # 32: the bit-sliced kernel
    want = _matrix_oracle(seqs)
    assert np.array_equal(M1, want) and np.array_equal(M2, want)


@pytest.mark.parametrize("rows", [4, 8, 16])
def test_preloaded_rows_choice_is_used_and_exact(rows):
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(72)
    pairs = [(rs.bases(int(m)), rs.bases(int(n))) for m, n in zip(rs.integers(1, 700, 50), rs.integers(1, 700, 50))]
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        ctx.set_autotune(True)
        nw.nw_align_batch(ctx, pool, off[0::2], lens[0::2], off[1::2], lens[1::2], (1, -1, -1), 0)
        key = [k for k in ctx.tuning() if k.startswith("batch_rows:")][0]
        ctx.set_tuning({key: rows})
        scores, cigars = nw.nw_align_batch(ctx, pool, off[0::2], lens[0::2], off[1::2], lens[1::2], (1, -1, -1),
                                           nw.NW_CIGAR)
        assert ctx.tuning()[key] == rows
    want = oracle.align_many(pairs)
    for k, (s, ops) in enumerate(want):
        assert scores[k] == s and cigars[k] == oracle.rle(ops), k


# The single-pair shape autotuner belongs to the scalar pair kernel; with
# s' = s - 2 gap in [0, 3] a pair runs on the bit-sliced stripes (one fixed
# shape), so these tests use a scoring outside that form.
SCALAR_SC = (2, -1, -2)


def test_bad_tuning_values_are_rejected():
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(73)
    a, b = rs.bases(3000), rs.bases(2900)
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        ctx.set_autotune(True)
        nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, SCALAR_SC, 0)
        key = [k for k in ctx.tuning() if k.startswith("pair_shape:")][0]
        ctx.set_tuning({key: 999})
        with pytest.raises(nw.NWError) as e:
            nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, SCALAR_SC, nw.NW_CIGAR)
        assert e.value.status == nw.NW_ERR_ARG
        # malformed lines are rejected by the library and change nothing
        before = ctx.tuning()
        assert nw.load().nw_ctx_set_tuning(ctx.handle, b"novalue\n") == nw.NW_ERR_ARG
        assert nw.load().nw_ctx_set_tuning(ctx.handle, b"k 12x\n") == nw.NW_ERR_ARG
        assert ctx.tuning() == before
        ctx.sync()


@pytest.mark.parametrize("m,n", [(3000, 2950), (700, 900), (5000, 300)])
def test_autotuned_single_pair_exact(m, n):
    import torch
    import paper_2412_21103_gb300 as nw
    p = seqgen.long_mutated_pair(m + n, m=m)
    a, b = p.a, p.b[:n] if n < p.b.size else p.b
    want_s, ops = oracle.align(a, b, *SCALAR_SC)
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        ctx.set_autotune(True)
        for _ in range(2):
            s, cig = nw.nw_align(ctx, nw.pack_codes(a), a.size, nw.pack_codes(b), b.size, SCALAR_SC, nw.NW_CIGAR)
            assert s == want_s and cig == oracle.rle(ops)
        keys = [k for k in ctx.tuning() if k.startswith("pair_shape:")]
        assert len(keys) == 1


def test_graph_replay_all_pairs_reads_current_pool():
    import torch
    import paper_2412_21103_gb300 as nw
    seqs = _family(74, 48)
    pool, off, lens = nw.pool_of(seqs)
    dpool = torch.from_numpy(pool).cuda()
    n = len(seqs)
    out = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        nw.nw_score_all_pairs(ctx, dpool, off, lens, (1, -1, -1), nw.NW_GRAPH, out)
        ctx.sync()
        first = out.cpu().numpy().copy()
        out.zero_()
        nw.nw_score_all_pairs(ctx, dpool, off, lens, (1, -1, -1), nw.NW_GRAPH, out)   # replay
        ctx.sync()
        second = out.cpu().numpy().copy()
        st = ctx.graph_stats()
        assert st["captures"] == 1 and st["replays"] == 1 and st["graphs"] == 1
        # same buffers and lengths, new bases: the replay computes the new matrix
        rs = seqgen.Stream(75)
        seqs2 = [rs.bases(s.size) for s in seqs]
        pool2, off2, lens2 = nw.pool_of(seqs2)
        assert np.array_equal(off2, off) and np.array_equal(lens2, lens)
        dpool.copy_(torch.from_numpy(pool2))
        nw.nw_score_all_pairs(ctx, dpool, off, lens, (1, -1, -1), nw.NW_GRAPH, out)
        ctx.sync()
        third = out.cpu().numpy().copy()
        assert ctx.graph_stats()["replays"] == 2
        # other lengths: a new capture, not a stale replay
        nw.nw_score_all_pairs(ctx, dpool, off[:-1], lens[:-1], (1, -1, -1), nw.NW_GRAPH, out)
        ctx.sync()
        assert ctx.graph_stats()["captures"] == 2
    want = _matrix_oracle(seqs)
    assert np.array_equal(first, want) and np.array_equal(second, want)
    assert np.array_equal(third, _matrix_oracle(seqs2))


def test_graph_replay_batch_scores():
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(76)
    pairs = [(rs.bases(int(m)), rs.bases(int(n))) for m, n in zip(rs.integers(1, 900, 300), rs.integers(1, 900, 300))]
    seqs = []
    for a, b in pairs:
        seqs += [a, b]
    pool, off, lens = nw.pool_of(seqs)
    dpool = torch.from_numpy(pool).cuda()
    scores = torch.zeros(len(pairs), dtype=torch.int32, device="cuda")
    want = oracle.score_many(pairs)
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        for k in range(3):
            scores.zero_()
            nw.nw_align_batch(ctx, dpool, off[0::2], lens[0::2], off[1::2], lens[1::2], (1, -1, -1), nw.NW_GRAPH,
                              scores)
            ctx.sync()
            assert scores.cpu().numpy().tolist() == want, k
        st = ctx.graph_stats()
        assert st["captures"] == 1 and st["replays"] == 2
        with pytest.raises(nw.NWError):
            nw.nw_align_batch(ctx, pool, off[0::2], lens[0::2], off[1::2], lens[1::2], (1, -1, -1), nw.NW_GRAPH)
        ctx.sync()


def test_graph_cache_evicts_and_stays_exact():
    """More distinct calls than the cache holds: old graphs are evicted (with
    their scratch), every result stays exact."""
    import torch
    import paper_2412_21103_gb300 as nw
    with nw.Context(0, torch.cuda.current_stream()) as ctx:
        for k in range(10):
            seqs = _family(80 + k, 12 + k)
            pool, off, lens = nw.pool_of(seqs)
            dpool = torch.from_numpy(pool).cuda()
            out = torch.zeros((len(seqs), len(seqs)), dtype=torch.int32, device="cuda")
            for _ in range(2):
                nw.nw_score_all_pairs(ctx, dpool, off, lens, (1, -1, -1), nw.NW_GRAPH, out)
            ctx.sync()
            assert np.array_equal(out.cpu().numpy(), _matrix_oracle(seqs)), k
        st = ctx.graph_stats()
        assert st["graphs"] == 8 and st["captures"] == 10 and st["replays"] == 10
