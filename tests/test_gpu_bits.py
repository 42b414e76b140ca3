"""GPU parity of the bit-sliced score-only kernel (rows per lane 32): the
difference form of the Sec. 2.3 recurrence, 32 cells per word, taken by
nw_score_all_pairs and score-only nw_align_batch whenever
0 <= s'(mismatch) <= s'(match) <= 3 with s' = s - 2*gap.  Scores must equal
the oracle's exactly: ragged and empty sequences, sequences at unaligned pool
offsets, lanes of one warp with very different shapes, every scoring the
kernel takes, and the scalar kernel for scorings it does not take."""
import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu

# (match, mismatch, gap): s'(match), s'(mismatch) = 3/1 (the paper's), 3/2, 2/1, 3/0, 1/1
BITS_SCORINGS = [(1, -1, -1), (1, 0, -1), (0, -1, -1), (1, -2, -1), (1, 1, 0)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream())
    c.set_profiling(True)
    yield c
    c.close()


def _bits_launches(c):
    return c.kernel_stats().get("bits_score", (0, 0.0))[0]


def _pool_unaligned(seqs, seed):
    """Pack sequences at irregular byte offsets (gaps of 0..5 bytes)."""
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(seed)
    offs, pos, chunks = [], 0, []
    for s in seqs:
        gap = int(rs.integers(0, 6, 1)[0])
        chunks.append(np.zeros(gap, np.uint8))
        pos += gap
        offs.append(pos)
        packed = nw.pack_codes(s) if s.size else np.zeros(0, np.uint8)
        chunks.append(packed)
        pos += packed.size
    chunks.append(np.zeros(64, np.uint8))
    return np.concatenate(chunks), np.array(offs, np.uint64), np.array([s.size for s in seqs], np.uint32)


def _oracle_matrix(seqs, sc):
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


def test_bits_scorings_are_the_ones_that_fit_two_planes():
    for m, x, g in BITS_SCORINGS:
        sm, sx = m - 2 * g, x - 2 * g
        assert 0 <= sx <= sm <= 3


@pytest.mark.parametrize("sc", BITS_SCORINGS)
def test_all_pairs_ragged_family_every_scoring(ctx, sc):
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(400 + sc[0] * 7 + sc[1] * 3)
    lens = [0, 1, 2, 3, 31, 32, 33, 63, 64, 65, 95, 96, 97, 100, 129, 200, 257, 300, 333]
    seqs = [rs.bases(L) for L in lens]
    root = rs.bases(600)
    seqs += [seqgen.mutate_distinct(root[: int(L)], rs, 0.15)[0] for L in rs.integers(100, 600, 12)]
    pool, off, ln = _pool_unaligned(seqs, 401)
    before = _bits_launches(ctx)
    M = nw.nw_score_all_pairs(ctx, pool, off, ln, sc)
    assert _bits_launches(ctx) == before + 1
    assert np.array_equal(M, _oracle_matrix(seqs, sc))


@pytest.mark.parametrize("sc", [(2, -1, -2), (1, -3, -1), (2, -1, -1)])
def test_scorings_beyond_two_planes_take_the_scalar_kernel(ctx, sc):
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(410 + sc[0])
    seqs = [rs.bases(int(L)) for L in rs.integers(0, 300, 14)]
    pool, off, ln = nw.pool_of(seqs)
    before = _bits_launches(ctx)
    M = nw.nw_score_all_pairs(ctx, pool, off, ln, sc)
    assert _bits_launches(ctx) == before
    assert np.array_equal(M, _oracle_matrix(seqs, sc))


def test_batch_lanes_of_very_different_shapes(ctx):
    """Pairs whose stripe counts and widths differ a lot (long x short,
    short x long, empty sides, equal stripe count with very different widths)
    share warps and jobs; every score equals the oracle's."""
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(420)
    shapes = [(0, 0), (0, 17), (17, 0), (1, 1), (1, 3000), (3000, 1), (40, 2500), (2500, 40), (33, 33),
              (64, 2000), (64, 5), (65, 1999), (1024, 1024), (1025, 31), (7, 7)]
    shapes += [(int(m), int(n)) for m, n in zip(rs.integers(1, 700, 60), rs.integers(1, 700, 60))]
    pairs = []
    for k, (m, n) in enumerate(shapes):
        a = rs.bases(m)
        if k % 2 and m and n:
            b = seqgen.mutate_distinct(np.resize(a, n), rs, 0.1)[0] if n <= m else rs.bases(n)
            b = b[:n] if b.size >= n else np.concatenate([b, rs.bases(n - b.size)])
        else:
            b = rs.bases(n)
        pairs.append((a, b))
    seqs = [s for p in pairs for s in p]
    pool, off, ln = _pool_unaligned(seqs, 421)
    before = _bits_launches(ctx)
    scores, _ = nw.nw_align_batch(ctx, pool, off[0::2], ln[0::2], off[1::2], ln[1::2], (1, -1, -1), 0)
    assert _bits_launches(ctx) == before + 1
    assert scores.tolist() == oracle.score_many(pairs, 1, -1, -1)


def test_device_buffers_and_graph_replay(ctx):
    """All-pairs on device buffers under NW_GRAPH: the captured bit-sliced
    launches replay with exact results, and a replay re-reads the pool."""
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(430)
    seqs = [rs.bases(int(L)) for L in rs.integers(50, 400, 24)]
    pool, off, ln = nw.pool_of(seqs)
    dpool = torch.from_numpy(pool).cuda()
    out = torch.zeros((len(seqs), len(seqs)), dtype=torch.int32, device="cuda")
    for _ in range(2):
        nw.nw_score_all_pairs(ctx, dpool, off, ln, (1, -1, -1), nw.NW_GRAPH, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), _oracle_matrix(seqs, (1, -1, -1)))
    seqs2 = [rs.bases(int(L)) for L in ln]
    pool2, off2, ln2 = nw.pool_of(seqs2)
    assert np.array_equal(off2, off) and np.array_equal(ln2, ln)
    dpool.copy_(torch.from_numpy(pool2))
    nw.nw_score_all_pairs(ctx, dpool, off, ln, (1, -1, -1), nw.NW_GRAPH, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), _oracle_matrix(seqs2, (1, -1, -1)))


def test_preloaded_bits_choice_maps_to_a_pointer_kernel_for_cigars(ctx):
    """A tuning entry of 32 rows per lane (the bit-sliced kernel) selects it
    for score-only calls; a CIGAR call of the same signature fills with the
    16-row pointer kernel instead, and both are exact."""
    import torch
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(440)
    pairs = [(rs.bases(int(m)), rs.bases(int(n))) for m, n in zip(rs.integers(1, 500, 40), rs.integers(1, 500, 40))]
    seqs = [s for p in pairs for s in p]
    pool, off, ln = nw.pool_of(seqs)
    with nw.Context(0, torch.cuda.current_stream()) as c2:
        c2.set_autotune(True)
        nw.nw_align_batch(c2, pool, off[0::2], ln[0::2], off[1::2], ln[1::2], (1, -1, -1), 0)
        key = [k for k in c2.tuning() if k.startswith("batch_rows:")][0]
        c2.set_tuning({key: 32})
        s1, _ = nw.nw_align_batch(c2, pool, off[0::2], ln[0::2], off[1::2], ln[1::2], (1, -1, -1), 0)
        s2, cig = nw.nw_align_batch(c2, pool, off[0::2], ln[0::2], off[1::2], ln[1::2], (1, -1, -1), nw.NW_CIGAR)
    want = oracle.align_many(pairs)
    assert s1.tolist() == [s for s, _ in want] and s2.tolist() == [s for s, _ in want]
    assert cig == [oracle.rle(ops) for _, ops in want]


def test_host_buffers_graph_replay(ctx):
    """All-pairs with host buffers under NW_GRAPH: the pool is copied to the
    context's device slot before every call, so a replay of the captured
    launches reads the new contents; results stay exact."""
    import paper_2412_21103_gb300 as nw
    rs = seqgen.Stream(450)
    seqs = [rs.bases(int(L)) for L in rs.integers(40, 350, 20)]
    pool, off, ln = nw.pool_of(seqs)
    before = ctx.graph_stats()
    for _ in range(2):
        M = nw.nw_score_all_pairs(ctx, pool, off, ln, (1, -1, -1), nw.NW_GRAPH)
        assert np.array_equal(M, _oracle_matrix(seqs, (1, -1, -1)))
    seqs2 = [rs.bases(int(L)) for L in ln]
    pool2, off2, ln2 = nw.pool_of(seqs2)
    assert np.array_equal(off2, off) and np.array_equal(ln2, ln)
    M2 = nw.nw_score_all_pairs(ctx, pool2, off, ln, (1, -1, -1), nw.NW_GRAPH)
    assert np.array_equal(M2, _oracle_matrix(seqs2, (1, -1, -1)))
    after = ctx.graph_stats()
    assert after["replays"] >= before["replays"] + 2
