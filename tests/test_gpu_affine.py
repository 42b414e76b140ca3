"""GPU parity of affine-gap global alignment (nw_affine_align_batch, Gotoh)
against the CPU oracle: scores and CIGARs bit-exact over ragged lengths,
every rows-per-lane shape and several scorings; open cost 0 equals the
linear batch; pointer waves under a small budget; device buffers; and the
2,000-pair affine workload of the benchmark, every pair."""
import numpy as np
import pytest

import oracle
import seqgen

pytestmark = pytest.mark.gpu

LENGTHS = [0, 1, 2, 31, 32, 33, 95, 96, 97, 255, 256, 257, 300, 513, 1000]


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
        if k % 3 == 0 and m > 1:
            p = seqgen.long_mutated_pair(seed * 100 + k, m=m)
            out.append((p.a, p.b))
        else:
            out.append((rs.bases(m), rs.bases(n)))
    return out


@pytest.mark.parametrize("rows", ["4", "8", "16"])
@pytest.mark.parametrize("sc", [(1, -1, -2, -1), (2, -3, -5, -2), (1, -2, -1, -1)])
def test_affine_every_shape(ctx, rows, sc, monkeypatch):
    import paper_2412_21103_gb300 as nw
    monkeypatch.setenv("NW_AFFINE_R", rows)
    pairs = _pairs(60 + int(rows) - sc[2], 70)
    pool, ao, al, bo, bl = _pool(pairs)
    scores, cigars = nw.nw_affine_align_batch(ctx, pool, ao, al, bo, bl, sc, nw.NW_CIGAR)
    want = oracle.affine_align_many(pairs, *sc)
    for k, (s, ops) in enumerate(want):
        assert int(scores[k]) == s and cigars[k] == oracle.rle(ops), k
    s_only, _ = nw.nw_affine_align_batch(ctx, pool, ao, al, bo, bl, sc, 0)
    assert s_only.tolist() == [s for s, _ in want]


def test_open_cost_zero_equals_the_linear_batch(ctx):
    import paper_2412_21103_gb300 as nw
    pairs = _pairs(99, 80)
    pool, ao, al, bo, bl = _pool(pairs)
    s1, c1 = nw.nw_affine_align_batch(ctx, pool, ao, al, bo, bl, (2, -1, 0, -2), nw.NW_CIGAR)
    s2, c2 = nw.nw_align_batch(ctx, pool, ao, al, bo, bl, (2, -1, -2), nw.NW_CIGAR)
    assert s1.tolist() == s2.tolist() and c1 == c2


def test_affine_waves_under_a_small_budget():
    import torch
    import paper_2412_21103_gb300 as nw
    c = nw.Context(0, torch.cuda.current_stream(), mem_budget=64 << 20)
    pairs = [(p.a, p.b) for p in (seqgen.long_mutated_pair(500 + k, m=2500 + 300 * k) for k in range(10))]
    pool, ao, al, bo, bl = _pool(pairs)
    scores, cigars = nw.nw_affine_align_batch(c, pool, ao, al, bo, bl, (2, -3, -5, -2), nw.NW_CIGAR)
    for k, (s, ops) in enumerate(oracle.affine_align_many(pairs, 2, -3, -5, -2)):
        assert int(scores[k]) == s and cigars[k] == oracle.rle(ops), k
    c.close()


def test_affine_workload_full_size_device_buffers(ctx):
    """The benchmark's workload (2,000 pairs, 1-5 kb, seed 1007, scoring
    2/-3/-5/-2) on device buffers: every score and CIGAR against the oracle."""
    import torch
    import paper_2412_21103_gb300 as nw
    pairs = [(p.a, p.b) for p in seqgen.band_pairs(1007, npairs=2000, lmin=1000, lmax=5000)]
    pool, ao, al, bo, bl = _pool(pairs)
    n = len(pairs)
    coff = nw._cigar_offsets(al, bl)
    scores = torch.zeros(n, dtype=torch.int32, device="cuda")
    cpool = torch.zeros(int(coff[-1]), dtype=torch.uint8, device="cuda")
    clen = torch.zeros(n, dtype=torch.int64, device="cuda")
    nw.nw_affine_align_batch(ctx, torch.from_numpy(pool).cuda(), ao, al, bo, bl, (2, -3, -5, -2), nw.NW_CIGAR,
                             scores, cpool, coff, clen)
    ctx.sync()
    cp, cl, sc = cpool.cpu().numpy(), clen.cpu().numpy(), scores.cpu().numpy()
    for k, (s, ops) in enumerate(oracle.affine_align_many(pairs, 2, -3, -5, -2)):
        assert int(sc[k]) == s, k
        assert cp[int(coff[k]): int(coff[k]) + int(cl[k])].tobytes().decode() == oracle.rle(ops), k
